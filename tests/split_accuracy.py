"""Measure the accuracy of the benchmark's split convolution (run on a machine with the GPU):

    python tests/split_accuracy.py [--out profiles/split_accuracy_nside2048.json]

The Planck-resolution workload (nside 2048, l_max 4096, 5' Gaussian beam, l_cut 1024,
theta_cut 240') on a Gaussian random field with C_l = 1/(l+10)^2 (seed family 2, the
accuracy field of the GPU tests): the fractional rms C_l error eps_C (Sec. 3) of [harmonic
part by the oracle's synthesis + GPU real-space part] against the full harmonic
convolution of the same field, split into the fitted kernel's own error (model) and the
pixel sum's (pix), for two readings of the cut:

  c1    the fitted real-space kernel reaches zero with zero slope at theta_cut (this
        library's default, KSC_CUT_C1: an addition to the paper's fit);
  free  the paper's fit as printed (Eq. 3-5, KSC_CUT_FREE): K_r may jump at the cut.

About 4 minutes of FP64 spherical-harmonic transforms on the host.  The result is a
measurement of the GPU path, written for bench.py to quote; no test reads it.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1409_4441_gb300 import inputs  # noqa: E402

ARC = inputs.ARCMIN
NSIDE, LMAX, FWHM, LCUT, TC = 2048, 4096, 5.0 * ARC, 1024, 240.0 * ARC


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "profiles",
                                                  "split_accuracy_nside2048.json"))
    args = ap.parse_args()
    import torch
    from paper_1409_4441_gb300 import ksconv as K

    ell = np.concatenate([np.arange(mm, LMAX + 1) for mm in range(LMAX + 1)])
    b = inputs.gaussian_beam(LMAX, FWHM)
    cl = inputs.cl_grf(LMAX)
    seed = inputs.seed_for(2)
    alm0 = inputs.grf_alm(LMAX, cl, seed)
    m = O.alm2map(NSIDE, alm0, LMAX).astype(np.float32)
    alm = O.map2alm(NSIDE, m.astype(np.float64), LMAX)
    cf = O.alm2cl(O.map2alm(NSIDE, O.alm2map(NSIDE, alm * b[ell], LMAX), LMAX), LMAX)
    x = torch.tensor(m, device="cuda")
    y = torch.empty_like(x)
    out = {"workload": "nside 2048, l_max 4096, 5' Gaussian beam, l_cut 1024, theta_cut 240'",
           "field": f"Gaussian random field, C_l = 1/(l+10)^2, seed {seed}",
           "metric": "fractional rms C_l error, l >= 2 (Sec. 3)",
           "command": "python tests/split_accuracy.py",
           "date": datetime.date.today().isoformat()}
    for name, cut in (("c1", K.KSC_CUT_C1), ("free", K.KSC_CUT_FREE)):
        with K.make_split(b, NSIDE, LCUT, TC, cl_in=cl, cut_continuity=cut) as sp:
            kh, kt = K.split_harmonic(sp), K.split_model(sp)
            eq6 = K.split_info(sp)["frac_error"]
            K.conv_real(sp, x, y)
            K.device_status(sp)
            real = y.cpu().numpy().astype(np.float64)
        kf = np.zeros(LMAX + 1)
        kf[: LCUT + 1] = kh
        split = O.alm2map(NSIDE, alm * kf[ell], LMAX) + real
        ideal = O.alm2map(NSIDE, alm * kt[ell], LMAX)
        cs = O.alm2cl(O.map2alm(NSIDE, split, LMAX), LMAX)
        ci = O.alm2cl(O.map2alm(NSIDE, ideal, LMAX), LMAX)
        out[name] = {"eps_C": O.eps_cl(cs, cf, lmin=2), "model": O.eps_cl(ci, cf, lmin=2),
                     "pix": O.eps_cl(cs, ci, lmin=2), "eq6_alpha5": eq6}
        print(name, out[name], flush=True)
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
