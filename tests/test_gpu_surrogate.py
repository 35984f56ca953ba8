"""The surrogate split selector: the library's CUDA forward / backward / Adam kernels
against the FP64 reference network, and what the trained network gains over the method
without it on measured splits (tests/golden/surrogate_splits.csv, written by
tests/surrogate_data.py).
"""
import os

import numpy as np
import pytest

from oracle import mlp as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DATA = os.path.join(os.path.dirname(__file__), "golden", "surrogate_splits.csv")


@pytest.fixture(scope="module")
def K():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_4441_gb300 import ksconv
    return ksconv


def _problem(n=150, seed=5):
    g = np.random.default_rng(seed)
    p = (g.normal(0.0, 0.25, M.N_PARAMS)).astype(np.float32)
    x = (g.normal(size=(n, 4)) * [1.0, 2.0, 0.5, 3.0] + [7.0, -6.0, 5.0, -2.0]).astype(np.float32)
    t = (g.normal(size=(n, 2)) * [0.7, 1.5] + [-5.0, 1.0]).astype(np.float32)
    norm = (np.array([7.0, -6.0, 5.0, -2.0], np.float32), np.array([1.0, 2.0, 0.5, 3.0], np.float32),
            np.array([-5.0, 1.0], np.float32), np.array([0.7, 1.5], np.float32))
    return p, x, t, norm


def test_forward_and_gradient_match_the_fp64_reference(K):
    """150 samples = two full 64-sample tiles and a ragged tail of 22."""
    p, x, t, norm = _problem()
    with K.MLP(seed=1) as net:
        net.set_params(p)
        net.set_norm(*norm)
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        y = net.predict(dx)
        torch.cuda.synchronize()
        g, loss = net.grad(dx, dt)
    y_ref, _ = M.forward(p.astype(np.float64), x, norm)
    loss_ref, g_ref = M.loss_and_grad(p.astype(np.float64), x, t, norm)
    np.testing.assert_allclose(y.cpu().numpy(), y_ref, rtol=2e-5, atol=2e-5 * np.abs(y_ref).max())
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    err = np.abs(g - g_ref)
    assert err.max() <= 1e-4 * np.abs(g_ref).max(), err.max() / np.abs(g_ref).max()


def test_one_training_step_is_the_adam_update(K):
    p, x, t, norm = _problem(n=70, seed=8)
    lr = 3e-3
    with K.MLP(seed=2) as net:
        net.set_params(p)
        net.set_norm(*norm)
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        net.train(dx, dt, epochs=2, lr=lr)
        got = net.get_params()
    q = p.astype(np.float64)
    m1 = np.zeros_like(q)
    m2 = np.zeros_like(q)
    for step in (1, 2):
        _, g = M.loss_and_grad(q, x, t, norm)
        q, m1, m2 = M.adam_step(q, g, m1, m2, step, lr)
    # FP32 kernels: each Adam step moves a parameter by about lr
    assert np.abs(got - q).max() <= 2e-2 * lr


def test_training_fits_a_smooth_function(K):
    g = np.random.default_rng(0)
    x = g.uniform(-1, 1, size=(600, 4)).astype(np.float32)
    t = np.stack([np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2], np.cos(x[:, 3]) - x[:, 0] ** 2],
                 axis=1).astype(np.float32)
    with K.MLP(seed=3) as net:
        net.set_norm(np.zeros(4), np.ones(4), t.mean(0), t.std(0))
        dx, dt = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        _, l0 = net.grad(dx, dt)
        l1 = net.train(dx, dt, epochs=1500, lr=3e-3)
    assert l1 < l0 / 100, (l0, l1)


def _load():
    rows = [ln.strip().split(",") for ln in open(DATA) if ln.strip() and not ln.startswith("#")]
    hdr = rows[0]
    d = {h: np.array([float(r[i]) for r in rows[1:]]) for i, h in enumerate(hdr)}
    return d


def _pick_by_net(pred, meas_ok, bound, margin, host):
    """Network's order: candidates predicted to clear the bound, cheapest first (cost =
    max(predicted GPU ms, host ms)), then the rest by predicted error; returns (trials
    until a measured pass, index, first choice)."""
    ok_pred = pred[:, 0] <= np.log10(bound) - margin
    pc = np.maximum(10.0 ** pred[:, 1].astype(np.float64), host)
    first = [i for i in np.argsort(pc, kind="stable") if ok_pred[i]]
    order = first + [i for i in np.argsort(pred[:, 0]) if not ok_pred[i]]
    for t, i in enumerate(order, 1):
        if meas_ok[i]:
            return t, i, (first[0] if first else -1)
    return len(order), None, (first[0] if first else -1)


@pytest.mark.skipif(not os.path.exists(DATA), reason="measured split data not generated")
def test_surrogate_choice_beats_the_eq6_choice_on_held_out_beams(K):
    """Train on the measured splits of most (nside, beam) groups; on held-out groups (two
    per nside), pick the cheapest split predicted to meet eps_C <= 1e-5 (0.2 decades of
    margin) and verify it with the measured run, stepping to the next candidate when the
    measurement rejects it.  Against (a) the method without the network, the Eq. 6
    estimate of Sec. 2: with the paper's alpha = 5, and with alpha refitted on the
    training data so the estimate bounds every measured error there, each taking the
    cheapest candidate the estimate accepts (measured costs); (b) a direct search running
    candidates cheapest first until one meets the bound.  A split's cost is max(measured
    GPU time, host time of the harmonic half) -- the halves run concurrently (Fig. 1) --
    with the host time from Eq. 8 spread over 16 cores.  The network must reach a split
    meeting the bound in every held-out group, at a total cost no higher than either Eq. 6
    choice (a group where Eq. 6 accepts nothing costs infinity: no split), with fewer trial
    runs than (b)."""
    d = _load()
    ARC = np.pi / (180 * 60)
    feats = K.split_features(d["nside"], d["fwhm_arcmin"] * ARC, d["l_cut"],
                             d["theta_cut_arcmin"] * ARC)
    targ = np.stack([np.log10(d["eps_c"]), np.log10(d["t_conv_ms"])], axis=1).astype(np.float32)
    groups = d["group"].astype(int)
    # held-out groups are drawn among those where some candidate of the grid meets the
    # bound when measured (no selector can succeed elsewhere: the narrowest beams, ~2.5
    # pixels, reach 1.1-2.4e-5 at best); every group stays in the training data
    feasible = {int(gg) for gg in np.unique(groups) if (d["eps_c"][groups == gg] <= 1e-5).any()}
    rng = np.random.default_rng(7)
    test_g = set()
    for ns in np.unique(d["nside"]):
        gs = np.array(sorted(set(groups[d["nside"] == ns].tolist()) & feasible))
        test_g |= set(int(v) for v in rng.choice(gs, size=2, replace=False))
    tr = np.array([gg not in test_g for gg in groups])
    bound, margin = 1e-5, 0.2
    with K.MLP(seed=11) as net:
        net.set_norm(feats[tr].mean(0), feats[tr].std(0), targ[tr].mean(0), targ[tr].std(0))
        dx = torch.tensor(feats[tr], device="cuda")
        dt = torch.tensor(targ[tr], device="cuda")
        loss = net.train(dx, dt, epochs=4000, lr=2e-3)
        sigma = d["eq6_alpha5"] / 5.0                   # Eq. 6 with alpha = 1
        alpha_fit = (d["eps_c"][tr] / sigma[tr]).max()  # bounds every training error
        tot = dict(net=0.0, eq6_paper=0.0, eq6_fit=0.0, net_trials=0, search_trials=0)
        lines = []
        for gg in sorted(test_g):
            sel = np.where(groups == gg)[0]
            meas_ok = d["eps_c"][sel] <= bound
            host = K.host_cost_ms(K.eq8_cost_model(cores=16), d["l_cut"][sel], d["lmax"][sel])
            cost = np.maximum(d["t_conv_ms"][sel], host)
            best, pred = net.select(feats[sel], np.log10(bound), margin=margin, host_ms=host)
            trials, pick, first = _pick_by_net(pred, meas_ok, bound, margin, host)
            assert best == first
            assert pick is not None, f"group {gg}: no candidate meets the bound"
            c_paper = min((c for c, s in zip(cost, sigma[sel]) if 5.0 * s <= bound), default=np.inf)
            c_fit = min((c for c, s in zip(cost, sigma[sel]) if alpha_fit * s <= bound),
                        default=np.inf)
            s_trials = int(np.argmax(meas_ok[np.argsort(cost)])) + 1
            tot["net"] += cost[pick]
            tot["eq6_paper"] += c_paper
            tot["eq6_fit"] += c_fit
            tot["net_trials"] += trials
            tot["search_trials"] += s_trials
            lines.append(f"  group {gg} nside {int(d['nside'][sel][0])}: net {cost[pick]:.2f} ms "
                         f"(eps {d['eps_c'][sel][pick]:.1e}, {trials} trial(s)); Eq.6 alpha 5 "
                         f"{c_paper:.2f} ms, refit {c_fit:.2f} ms; search {s_trials} trials")
    print(f"\nsurrogate: training loss {loss:.3g}, Eq. 6 alpha refit {alpha_fit:.3g} "
          f"(paper: 5)\n" + "\n".join(lines) +
          f"\n  total: net {tot['net']:.2f} ms, Eq.6 alpha 5 {tot['eq6_paper']:.2f} ms, refit "
          f"{tot['eq6_fit']:.2f} ms; trials net {tot['net_trials']} vs search "
          f"{tot['search_trials']}")
    assert tot["net"] <= tot["eq6_fit"] and tot["net"] <= tot["eq6_paper"]
    assert tot["net_trials"] < tot["search_trials"]


@pytest.mark.slow
@pytest.mark.skipif(not os.path.exists(DATA), reason="measured split data not generated")
def test_surrogate_chosen_split_at_nside4096(K):
    """One nside-4096 map (201M pixels), 3' beam, l_max 8192: the network trained on all
    measured splits picks (l_cut, theta_cut) from a grid for eps_C <= 1e-5 (0.2 decades of
    margin); the split is built, the map convolved on the GPU (timed), and sampled output
    pixels checked against the FP64 oracle with the same tabulated kernel."""
    import oracle as O
    from paper_1409_4441_gb300 import inputs
    d = _load()
    ARC = np.pi / (180 * 60)
    feats = K.split_features(d["nside"], d["fwhm_arcmin"] * ARC, d["l_cut"],
                             d["theta_cut_arcmin"] * ARC)
    targ = np.stack([np.log10(d["eps_c"]), np.log10(d["t_conv_ms"])], axis=1).astype(np.float32)
    nside, lmax, fwhm = 4096, 8192, 3.0 * ARC
    cands = [(lc, k * fwhm) for lc in (1024, 1536, 2048, 3072, 4096) for k in (16, 24, 32, 48, 64)]
    cf = K.split_features(np.full(len(cands), nside), np.full(len(cands), fwhm),
                          [c[0] for c in cands], [c[1] for c in cands])
    host = K.host_cost_ms(K.eq8_cost_model(cores=16), [c[0] for c in cands], lmax)
    with K.MLP(seed=12) as net:
        net.set_norm(feats.mean(0), feats.std(0), targ.mean(0), targ.std(0))
        net.train(torch.tensor(feats, device="cuda"), torch.tensor(targ, device="cuda"),
                  epochs=4000, lr=2e-3)
        best, pred = net.select(cf, -5.0, margin=0.2, host_ms=host)
    assert best >= 0
    lcut, tc = cands[best]
    b = inputs.gaussian_beam(lmax, fwhm)
    with K.make_split(b, nside, lcut, tc, cl_in=inputs.cl_grf(lmax)) as sp:
        info = K.split_info(sp)
        m = inputs.white_noise_map(nside, inputs.seed_for(5, 4096)).astype(np.float32)
        x = torch.tensor(m, device="cuda")
        y = torch.empty_like(x)
        K.conv_real(sp, x, y)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        K.conv_real(sp, x, y)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        K.device_status(sp)
        got = y.cpu().numpy().astype(np.float64)
        n_int = info["n_intervals"]
        c_real = K.split_real_coeffs(sp)
    npix = 12 * nside * nside
    pairs = npix * npix * (1 - np.cos(tc)) / 2  # in-disc pairs, area estimate
    print(f"\nnside 4096: surrogate chose l_cut {lcut}, theta_cut {tc / ARC:.0f}' (predicted "
          f"log10 eps {pred[best, 0]:.2f}, host half {host[best]:.0f} ms by Eq. 8 on 16 cores); "
          f"Eq. 6 estimate {info['frac_error']:.2e}; GPU {ms:.0f} ms per map = {1e3 / ms:.2f} "
          f"maps/s, {pairs / ms * 1e3:.3g} pairs/s")
    pix = inputs.sample_pixels(nside, 64, 41)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c_real, tc, n_int),
                            out_pix=pix)
    rms = np.sqrt(np.mean(ref ** 2))
    assert np.all(np.abs(got[pix] - ref) <= 1e-6 * rms + amb)


@pytest.mark.skipif(not os.path.exists(DATA), reason="measured split data not generated")
def test_selection_chain_falls_back_to_the_scan_and_a_measured_judge(K):
    """The selection chain of the surrogate (the network first, the Sec. 2 scan as the
    fallback, a measured run as the arbiter) on a beam outside the network's confident
    range: nside 128, a 110' beam (four pixel widths, inside the training beams), l_max
    256; the network asked for 1e-5 with a margin of five decades accepts nothing (-1),
    so the scan (ksc_scan_split: theta_cut 600'-3600' in 300' steps, l_cut searched, Eq. 6
    with alpha refitted to bound every training error) proposes splits in cost order and
    each is judged by its measured eps_C (GPU real-space part + the oracle's harmonic half
    against the full harmonic convolution of a GRF) until one passes, within three
    trials."""
    import oracle as O
    from paper_1409_4441_gb300 import inputs
    d = _load()
    ARC = np.pi / (180 * 60)
    feats = K.split_features(d["nside"], d["fwhm_arcmin"] * ARC, d["l_cut"],
                             d["theta_cut_arcmin"] * ARC)
    targ = np.stack([np.log10(d["eps_c"]), np.log10(d["t_conv_ms"])], axis=1).astype(np.float32)
    alpha = 5.0 * float((d["eps_c"] / d["eq6_alpha5"]).max())
    nside, lmax, fwhm, bound = 128, 256, 110.0 * ARC, 1e-5
    cands = [(lc, k * fwhm) for lc in (32, 64, 96, 128) for k in (16, 24, 32)]
    cf = K.split_features(np.full(len(cands), nside), np.full(len(cands), fwhm),
                          [c[0] for c in cands], [c[1] for c in cands])
    with K.MLP(seed=13) as net:
        net.set_norm(feats.mean(0), feats.std(0), targ.mean(0), targ.std(0))
        net.train(torch.tensor(feats, device="cuda"), torch.tensor(targ, device="cuda"),
                  epochs=1500, lr=2e-3)
        best, _ = net.select(cf, np.log10(bound), margin=5.0)
    assert best == -1
    # fallback: the scan over theta_cut with l_cut searched
    b = inputs.gaussian_beam(lmax, fwhm)
    cl = inputs.cl_grf(lmax)
    _, rows = K.scan_split(b, nside, cl_in=cl, theta_lo=600 * ARC, theta_hi=3600 * ARC,
                           theta_step=300 * ARC, bound=bound, alpha=alpha)
    order = sorted((r for r in rows if r["l_cut"] >= 0),
                   key=lambda r: max(r["t_gpu_ms"], r["t_host_ms"]))
    assert order, "the scan must propose a split"
    # the arbiter: measured eps_C of each proposal, cheapest first
    ell = np.concatenate([np.arange(mm, lmax + 1) for mm in range(lmax + 1)])
    alm0 = inputs.grf_alm(lmax, cl, inputs.seed_for(5, 9000))
    m = O.alm2map(nside, alm0, lmax).astype(np.float32)
    alm = O.map2alm(nside, m.astype(np.float64), lmax)
    cfull = O.alm2cl(O.map2alm(nside, O.alm2map(nside, alm * b[ell], lmax), lmax), lmax)
    x = torch.tensor(m, device="cuda")
    y = torch.empty_like(x)
    trials, passed = 0, None
    for r in order[:3]:
        trials += 1
        with K.make_split(b, nside, r["l_cut"], r["theta_cut"], cl_in=cl) as sp:
            kh = K.split_harmonic(sp)
            K.conv_real(sp, x, y)
            K.device_status(sp)
            real = y.cpu().numpy().astype(np.float64)
        kf = np.zeros(lmax + 1)
        kf[: r["l_cut"] + 1] = kh
        cs = O.alm2cl(O.map2alm(nside, O.alm2map(nside, alm * kf[ell], lmax) + real, lmax), lmax)
        eps = O.eps_cl(cs, cfull, lmin=2)
        print(f"\nchain: scan proposal l_cut {r['l_cut']} theta {r['theta_cut'] / ARC:.0f}': "
              f"Eq.6 (refit) {r['error']:.1e}, measured eps_C {eps:.1e}")
        if eps <= bound:
            passed = r
            break
    assert passed is not None, f"no scan proposal passed in {trials} trials"
