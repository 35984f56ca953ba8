"""GPU parity of the real-space convolution (the hot path) against the FP64 oracle.

Tolerance (per output pixel): |gpu - oracle| <= 1e-6 * rms(oracle) + ambig, where
ambig bounds pairs whose chord^2 lies within 1e-6 (relative) of the cut, which
FP32 and FP64 may legitimately classify differently.  Maps are rounded to FP32
before both sides see them.
"""
import numpy as np
import pytest

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
    assert torch.cuda.is_available()
    return ksconv


def _run(K, sp, m32):
    x = torch.tensor(m32, device="cuda")
    y = torch.full_like(x, float("nan"))
    K.conv_real(sp, x, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _check(got, ref, amb, rel=1e-6):
    rms = np.sqrt(np.mean(ref ** 2))
    err = np.abs(got - ref)
    bad = err > rel * rms + amb
    assert not np.any(np.isnan(got))
    assert not bad.any(), (f"{bad.sum()} pixels over tolerance; max err {err.max():.3e}, "
                           f"rms {rms:.3e}")
    return err.max() / rms


def test_table_matches_oracle_legendre_sum(K):
    lmax, nside = 1535, 512
    tc = 90 * ARC
    c = inputs.gaussian_beam(lmax, 20 * ARC)
    c[:257] = 0.0
    with K.make_split_real(c, nside, tc) as sp:
        info = K.split_info(sp)
        tab = K.split_table(sp).astype(np.float64)
    n_int = info["n_intervals"]
    dc = O.chord_cut(tc)
    assert info["chord_cut"] == pytest.approx(dc, rel=1e-15)
    d = np.random.default_rng(3).uniform(0, dc, 50000)
    h = dc / n_int
    k = np.minimum((d / h).astype(int), n_int - 1)
    t = d / h - k
    a = tab[k]
    lib = a[:, 0] + t * (a[:, 1] + t * (a[:, 2] + t * a[:, 3]))
    tK, tD = O.hermite_nodes(c, tc, n_int)
    orc = O.hermite_eval(tK, tD, tc, d)
    exact = O.legendre_sum(c, 1 - d * d / 2)
    peak = np.abs(exact).max()
    assert np.abs(lib - orc).max() <= 2e-7 * peak
    assert np.abs(lib - exact).max() <= 3e-7 * peak


@pytest.mark.parametrize("cap_kernel", [0, 1])
@pytest.mark.parametrize("exact_weights", [0, 1])
@pytest.mark.parametrize("nside,tc_deg,lmax,fwhm_deg", [
    (1, 60.0, 3, 40.0),      # twelve pixels, several per disc
    (8, 180.0, 23, 10.0),    # whole sphere: every input ring, full-ring windows
    (16, 20.0, 47, 6.0),     # caps and belt, ragged 256-pixel chunks
    (32, 0.5, 95, 3.0),      # disc smaller than a pixel: only the self pair
    (64, 6.0, 191, 2.0),     # the 2-degree nside-64 workload (3 x FWHM cut)
])
def test_full_map_parity(K, nside, tc_deg, lmax, fwhm_deg, exact_weights, cap_kernel):
    """Both weight paths of the cap gather (tables in |N|, default, and the exact
    double-float chord for every pair), each summed by both cap kernels (FP32 FFMAs,
    default, and the tensor cores)."""
    tc = np.radians(tc_deg)
    c = inputs.gaussian_beam(lmax, np.radians(fwhm_deg))
    m = inputs.white_noise_map(nside, inputs.seed_for(1, nside)).astype(np.float32)
    with K.make_split_real(c, nside, tc, exact_weights=exact_weights,
                           cap_kernel=cap_kernel) as sp:
        n_int = K.split_info(sp)["n_intervals"]
        got = _run(K, sp, m)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int))
    _check(got, ref, amb)
    # against the exact kernel too (table interpolation error included)
    ex, amb2 = O.brute_conv(nside, m.astype(np.float64), tc, c=c)
    _check(got, ex, amb2, rel=2e-6)


@pytest.mark.parametrize("nside,lmax,lcut,tc_deg,fwhm_deg", [
    (128, 383, 64, 4.0, 1.0),    # oscillating high-pass remainder, caps of 127 rings
    (256, 767, 192, 2.0, 0.5),   # longer rings: table cells stretched to fit
])
def test_dphi_tables_match_exact_weights(K, nside, lmax, lcut, tc_deg, fwhm_deg):
    """The cap gather's dphi weight tables against exact per-pair weights: the tables'
    interpolation error (at most 3e-7 of the kernel's peak per weight, rms ~1e-8) leaves
    the two paths within the per-pixel parity tolerance (1e-6 of the output rms) of each
    other; what remains is mostly the FP32 rounding of the largest outputs (a few ulp)."""
    tc = np.radians(tc_deg)
    c = inputs.gaussian_beam(lmax, np.radians(fwhm_deg))
    c[: lcut + 1] = 0.0
    m = inputs.white_noise_map(nside, inputs.seed_for(1, 1000 + nside)).astype(np.float32)
    with K.make_split_real(c, nside, tc) as a, K.make_split_real(c, nside, tc,
                                                                 exact_weights=1) as b:
        ya, yb = _run(K, a, m), _run(K, b, m)
        assert K.split_info(a)["frac_tabulated"] > 0.9
        assert K.split_info(b)["frac_tabulated"] == 0.0
    rms = np.sqrt(np.mean(yb ** 2))
    assert np.abs(ya - yb).max() <= 1e-6 * rms
    assert np.sqrt(np.mean((ya - yb) ** 2)) <= 1e-7 * rms


@pytest.mark.parametrize("nside,lmax,lcut,tc_deg,fwhm_deg", [
    (256, 767, 192, 2.0, 0.5),   # oscillating high-pass remainder, many cap ring pairs
    (128, 383, 0, 12.0, 3.0),    # wide windows: several staged segments per ring pair
])
def test_tensor_caps_match_ffma_caps(K, nside, lmax, lcut, tc_deg, fwhm_deg):
    """The cap ring pairs summed on the tensor cores (three-way BF16 splits, six MMAs
    per 16 positions, a fresh accumulator per step) and by the FP32 FFMA gather with
    the same weights: each within the per-pixel parity tolerance of the oracle on
    sampled pixels, and the two within the sum of those tolerances of each other
    everywhere (independent FP32 summation orders: a few ulp of the largest outputs)."""
    tc = np.radians(tc_deg)
    c = inputs.gaussian_beam(lmax, np.radians(fwhm_deg))
    c[: lcut + 1] = 0.0
    m = inputs.white_noise_map(nside, inputs.seed_for(1, 2000 + nside)).astype(np.float32)
    with K.make_split_real(c, nside, tc, cap_kernel=1) as a, \
            K.make_split_real(c, nside, tc) as b:
        ya, yb = _run(K, a, m), _run(K, b, m)
        K.device_status(a)
        n_int = K.split_info(a)["n_intervals"]
    pix = inputs.sample_pixels(nside, 1500, 29)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int),
                            out_pix=pix)
    _check(ya[pix], ref, amb)
    _check(yb[pix], ref, amb)
    rms = np.sqrt(np.mean(yb ** 2))
    assert np.abs(ya - yb).max() <= 2e-6 * rms
    # each path's FP32 summation error is about 1e-7 of the rms (rms over pixels)
    assert np.sqrt(np.mean((ya - yb) ** 2)) <= 2e-7 * rms


def test_self_pair_only(K):
    nside = 32
    tc = np.radians(0.5)
    c = inputs.gaussian_beam(95, np.radians(3.0))
    m = inputs.white_noise_map(nside, 99).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        got = _run(K, sp, m)
        tab = K.split_table(sp)
    k0 = float(tab[0, 0])
    np.testing.assert_allclose(got, m * k0 * np.float32(4 * np.pi / O.npix(nside)), rtol=1e-6)


def test_high_pass_kernel_parity_nside256(K):
    """An oscillating real-space remainder (l > l_cut of a beam) at 256-pixel chunks
    over many rings, full map against the tabulated-kernel oracle."""
    nside, lmax, lcut = 128, 383, 64
    tc = np.radians(4.0)
    c = inputs.gaussian_beam(lmax, np.radians(1.0))
    c[: lcut + 1] = 0.0
    m = inputs.white_noise_map(nside, 5).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        n_int = K.split_info(sp)["n_intervals"]
        got = _run(K, sp, m)
    pix = inputs.sample_pixels(nside, 3000, 17)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int),
                            out_pix=pix)
    _check(got[pix], ref, amb)


@pytest.mark.parametrize("tc_arcmin", [240.0])
def test_nside2048_sampled_parity(K, tc_arcmin):
    """The Planck-resolution workload (nside 2048, l_max 4096, 5' beam high-passed at
    l_cut 1024, theta_cut 240'), same launch as the benchmark, checked on sampled
    output pixels."""
    nside, lmax, lcut = 2048, 4096, 1024
    tc = tc_arcmin * ARC
    c = inputs.gaussian_beam(lmax, 5 * ARC)
    c[: lcut + 1] = 0.0
    m = inputs.white_noise_map(nside, inputs.seed_for(3)).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        info = K.split_info(sp)
        n_int = info["n_intervals"]
        got = _run(K, sp, m)
    # nearly every cap weight comes from a dphi table at this geometry (the rest:
    # whole-ring windows at the poles)
    assert info["frac_tabulated"] >= 0.99
    pix = inputs.sample_pixels(nside, 200, 23)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int),
                            out_pix=pix)
    _check(got[pix], ref, amb)


def test_nside2048_worst_pixels(K):
    """The same workload over the whole map: the pixels where the table path and the
    exact-weight path (exact_weights = 1) differ most are where FP32 rounding is largest.
    Both paths must be within tolerance of the oracle there, with the rms taken over
    sampled pixels."""
    nside, lmax, lcut = 2048, 4096, 1024
    tc = 240 * ARC
    c = inputs.gaussian_beam(lmax, 5 * ARC)
    c[: lcut + 1] = 0.0
    m = inputs.white_noise_map(nside, inputs.seed_for(3)).astype(np.float32)
    got = []
    for ew in (0, 1):
        with K.make_split_real(c, nside, tc, exact_weights=ew) as sp:
            n_int = K.split_info(sp)["n_intervals"]
            got.append(_run(K, sp, m))
    worst = np.argsort(np.abs(got[0] - got[1]))[::-1][:24]
    pix = np.concatenate([inputs.sample_pixels(nside, 200, 29), worst])
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int),
                            out_pix=pix)
    rms = np.sqrt(np.mean(ref[:200] ** 2))
    for g in got:
        err = np.abs(g[pix] - ref)
        assert (err <= 1e-6 * rms + amb).all(), (err.max() / rms, pix[np.argmax(err)])


def test_bands_multimap_host_bitwise_and_batch(K):
    nside = 32
    tc = np.radians(8.0)
    c = inputs.gaussian_beam(95, np.radians(3.0))
    maps = np.stack([inputs.white_noise_map(nside, 40 + i) for i in range(3)]).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        x = torch.tensor(maps, device="cuda")
        full = torch.empty_like(x)
        for i in range(3):
            K.conv_real(sp, x[i], full[i])
        # latitude bands, written into one output in several calls
        band = torch.full_like(x[0], float("nan"))
        nr = 4 * nside - 1
        for lo, hi in [(1, 17), (18, 64), (65, nr)]:
            K.conv_real_rings(sp, x[0], band, lo, hi)
        mm = torch.empty_like(x)
        K.conv_real_multimap(sp, x, mm, 3)
        torch.cuda.synchronize()
        host = K.conv_real_host(sp, maps[1])
        assert torch.equal(band, full[0])
        assert torch.equal(mm, full)
        assert np.array_equal(host, full[1].cpu().numpy())
    # ragged batch of different nsides / kernels
    specs = [(8, 20.0, 23, 8.0), (16, 12.0, 47, 4.0), (32, 8.0, 95, 3.0)]
    sps, ins, outs, singles = [], [], [], []
    for ns, td, lm, fw in specs:
        cc = inputs.gaussian_beam(lm, np.radians(fw))
        sps.append(K.make_split_real(cc, ns, np.radians(td)))
        ins.append(torch.tensor(inputs.white_noise_map(ns, ns).astype(np.float32), device="cuda"))
        outs.append(torch.empty_like(ins[-1]))
        singles.append(torch.empty_like(ins[-1]))
        K.conv_real(sps[-1], ins[-1], singles[-1])
    K.conv_real_batch(sps, ins, outs)
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):  # batch kernels: equal to FP32 rounding
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        assert np.abs(a - b).max() <= 1e-6 * np.sqrt(np.mean(b ** 2))
    for s in sps:
        s.close()


def test_pair_count_matches_oracle(K):
    nside = 32
    tc = np.radians(7.3)
    c = inputs.gaussian_beam(95, np.radians(3.0))
    with K.make_split_real(c, nside, tc) as sp:
        n = K.count_pairs(sp)
        assert K.split_info(sp)["n_pairs"] == n
    cnt = O.count_pairs(nside, tc)
    _, amb = O.brute_conv(nside, np.ones(O.npix(nside)), tc, c=np.array([4 * np.pi]), amb_eps=1e-6)
    n_amb = int(round(amb.sum() / (4 * np.pi / O.npix(nside))))
    assert abs(n - cnt.sum()) <= n_amb


@pytest.mark.parametrize("nside,tc_deg,lmax,fwhm_deg", [
    (1, 90.0, 3, 40.0), (2, 45.0, 7, 20.0), (4, 100.0, 11, 20.0), (8, 180.0, 23, 10.0),
    (16, 3.0, 47, 1.5), (32, 30.0, 95, 3.0), (128, 4.0, 383, 1.0),
])
def test_fast_path_matches_general_path(K, nside, tc_deg, lmax, fwhm_deg):
    """Circulant belt kernel + symmetric gather (default) against the general
    ring-pair gather: same sums in a different order."""
    tc = np.radians(tc_deg)
    c = inputs.gaussian_beam(lmax, np.radians(fwhm_deg))
    m = inputs.white_noise_map(nside, 77 + nside).astype(np.float32)
    outs = []
    for path in (0, 1):
        with K.make_split_real(c, nside, tc, path=path) as sp:
            assert K.split_info(sp)["path"] == path or nside >= 8 and tc_deg > 90
            outs.append(_run(K, sp, m))
            K.device_status(sp)
    rms = np.sqrt(np.mean(outs[1] ** 2))
    assert np.abs(outs[0] - outs[1]).max() <= 1e-6 * rms


def test_stages_compose_bitwise_and_counts(K):
    nside = 64
    tc = np.radians(12.0)
    c = inputs.gaussian_beam(191, np.radians(2.0))
    m = torch.tensor(inputs.white_noise_map(nside, 3).astype(np.float32), device="cuda")
    with K.make_split_real(c, nside, tc) as sp:
        a = torch.empty_like(m); b = torch.empty_like(m)
        K.conv_real(sp, m, a)
        K.conv_real_stage(sp, m, b, 1)
        K.conv_real_stage(sp, m, b, 2)
        K.device_status(sp)
        assert torch.equal(a, b)
        n = K.count_pairs(sp)
        info = K.split_info(sp)
    cnt = O.count_pairs(nside, tc)
    assert abs(n - cnt.sum()) <= 8
    # belt-belt pairs: both pixels with |z| <= 2/3
    z = O.pix2vec(nside)[:, 2]
    belt = np.abs(z) <= 2 / 3 + 1e-12
    assert 0 < info["n_pairs_belt"] < n
    assert abs(info["n_pairs_belt"] - O.count_pairs(nside, tc, out_pix=np.where(belt)[0]).sum()) \
        <= abs(n - info["n_pairs_belt"])  # sanity: belt outputs dominate belt-belt pairs


def test_bounded_wait_runs_out_and_context_survives(K):
    """Failure detection without a fault: a bounded mbarrier wait that nothing
    completes runs out, the CTA raises the split's device error flag and returns; the
    host reads KSC_ERR_TIMEOUT once (the flag is cleared), and the same context then
    convolves a map within the oracle parity."""
    nside = 16
    tc = np.radians(20.0)
    c = inputs.gaussian_beam(47, np.radians(6.0))
    m = inputs.white_noise_map(nside, 77).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        K.probe_wait_timeout(sp, max_polls=1 << 12)  # runs out in well under a second
        with pytest.raises(K.KsconvError) as e:
            K.device_status(sp)
        assert e.value.code == K.KSC_ERR_TIMEOUT
        K.device_status(sp)  # cleared
        n_int = K.split_info(sp)["n_intervals"]
        got = _run(K, sp, m)
        K.device_status(sp)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int))
    _check(got, ref, amb)
