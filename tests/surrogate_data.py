"""Measure splits for the surrogate's training set (run on a machine with the GPU):

    python tests/surrogate_data.py [--out tests/golden/surrogate_splits.csv] [--groups 128:36,256:24,512:10]

For each (nside, beam) group: one Gaussian random field with C_l = 1/(l+10)^2 up to
l_max = 2 nside and its full harmonic convolution (oracle SHT); then for every (l_cut,
theta_cut) on a grid: the least-squares split (library, default C1 cut), the GPU real-space
convolution timed with CUDA events (median of three), and eps_C of the split convolution
against the full one (Sec. 3's fractional rms C_l error; harmonic half by the oracle
synthesis).  Beams are drawn uniformly in [2.5, 8] pixel widths, theta_cut in 16..64 beam
widths (at most 60 degrees), l_cut in l_max/8 .. l_max/2: the pixel-scale shape of the
Planck-resolution workload.  Columns are described in the file's header.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1409_4441_gb300 import inputs  # noqa: E402

ARC = inputs.ARCMIN
LCUT_FRAC = (0.125, 0.1875, 0.25, 0.3125, 0.375, 0.5)
TC_FWHM = (16, 24, 32, 40, 48, 56, 64)
COLUMNS = ("group", "nside", "lmax", "fwhm_arcmin", "l_cut", "theta_cut_arcmin", "eps_c",
           "eps_model", "eq6_alpha5", "t_conv_ms")


def measure(K, torch, nside, fwhm, group, out_rows):
    lmax = 2 * nside
    ell = np.concatenate([np.arange(mm, lmax + 1) for mm in range(lmax + 1)])
    b = inputs.gaussian_beam(lmax, fwhm)
    cl = inputs.cl_grf(lmax)
    alm0 = inputs.grf_alm(lmax, cl, inputs.seed_for(5, group))
    m = O.alm2map(nside, alm0, lmax).astype(np.float32)
    alm = O.map2alm(nside, m.astype(np.float64), lmax)
    full = O.alm2map(nside, alm * b[ell], lmax)
    cf = O.alm2cl(O.map2alm(nside, full, lmax), lmax)
    c_alm = O.alm2cl(alm, lmax)
    x = torch.tensor(m, device="cuda")
    y = torch.empty_like(x)
    st = torch.cuda.current_stream()
    for fr in LCUT_FRAC:
        lcut = int(round(fr * lmax))
        for k in TC_FWHM:
            tc = k * fwhm
            if tc > np.radians(60.0):
                continue
            with K.make_split(b, nside, lcut, tc, cl_in=cl) as sp:
                info = K.split_info(sp)
                kh, kt = K.split_harmonic(sp), K.split_model(sp)
                K.conv_real(sp, x, y)
                ts = []
                for _ in range(3):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    K.conv_real(sp, x, y)
                    e1.record(st)
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                K.device_status(sp)
                real = y.cpu().numpy().astype(np.float64)
            kf = np.zeros(lmax + 1)
            kf[: lcut + 1] = kh
            split = O.alm2map(nside, alm * kf[ell], lmax) + real
            cs = O.alm2cl(O.map2alm(nside, split, lmax), lmax)
            # the fitted kernel applied harmonically against the full kernel: the spectra
            # of alm K~_l and alm b_l exactly (no transform)
            out_rows.append((group, nside, lmax, fwhm / ARC, lcut, tc / ARC,
                             O.eps_cl(cs, cf, lmin=2),
                             O.eps_cl(kt ** 2 * c_alm, b ** 2 * c_alm, lmin=2),
                             info["frac_error"], float(np.median(ts))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "surrogate_splits.csv"))
    ap.add_argument("--groups", default="128:36,256:24,512:10",
                    help="(nside, beam groups) pairs: nside:count,...")
    args = ap.parse_args()
    import torch
    import __graft_entry__
    __graft_entry__.build()
    O.build()
    from paper_1409_4441_gb300 import ksconv as K
    rows = []
    group = 0
    t0 = time.time()
    for spec in args.groups.split(","):
        nside, count = (int(v) for v in spec.split(":"))
        pix = np.sqrt(4 * np.pi / (12 * nside * nside))
        draws = inputs.rng(inputs.seed_for(5, 1000 + nside)).uniform(2.5, 8.0, count)
        for w in draws:
            measure(K, torch, nside, w * pix, group, rows)
            print(f"group {group} nside {nside} fwhm {w * pix / ARC:.1f}' rows {len(rows)} "
                  f"({time.time() - t0:.0f} s)", flush=True)
            group += 1
    with open(args.out, "w") as f:
        f.write("# Measured splits for the surrogate split selector, written by tests/surrogate_data.py\n")
        f.write("# on a GB300: GRF input (C_l = 1/(l+10)^2, l_max = 2 nside), least-squares split with\n")
        f.write("# the C1 cut; eps_c = fractional rms C_l error of harmonic part (oracle synthesis) +\n")
        f.write("# GPU real-space part against the full harmonic convolution (Sec. 3); eps_model = the\n")
        f.write("# fitted kernel applied harmonically (exact spectra); eq6_alpha5 = the Eq. 6 estimate\n")
        f.write("# with alpha 5; t_conv_ms = GPU time of the real-space convolution (CUDA events,\n")
        f.write("# median of 3).\n")
        f.write(",".join(COLUMNS) + "\n")
        for r in rows:
            f.write(f"{r[0]},{r[1]},{r[2]},{r[3]:.6f},{r[4]},{r[5]:.6f},{r[6]:.6e},{r[7]:.6e},"
                    f"{r[8]:.6e},{r[9]:.6f}\n")
    print(f"wrote {len(rows)} rows to {args.out}")


if __name__ == "__main__":
    main()
