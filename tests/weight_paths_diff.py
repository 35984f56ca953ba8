"""Whole-map difference between the cap gather's two weight paths (run on a machine with the
GPU):

    python tests/weight_paths_diff.py

The nside-2048 benchmark split (l_max 4096, 5' Gaussian beam, l_cut 1024, theta_cut 240')
on the benchmark's white-noise map, convolved twice: with the odd-step weight tables
(default) and with every weight from the exact chord (exact_weights = 1).  The two differ
only in the cap gather's weights and in rounding.  Prints the maximum, the 99.99th
percentile and the mean of |table - exact| over the output rms, and the pixels where the
difference is largest (the candidates that test_nside2048_worst_pixels checks against the
oracle).  About a minute; no test reads the output.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    from paper_1409_4441_gb300 import inputs, ksconv as K

    arc = inputs.ARCMIN
    nside, lmax, lcut, tc = 2048, 4096, 1024, 240 * arc
    b = inputs.gaussian_beam(lmax, 5 * arc)
    cl = inputs.cl_grf(lmax)
    m = inputs.white_noise_map(nside, inputs.seed_for(3, 0)).astype(np.float32)
    x = torch.tensor(m, device="cuda")
    outs = []
    for ew in (0, 1):
        with K.make_split(b, nside, lcut, tc, cl_in=cl, exact_weights=ew) as sp:
            y = torch.empty_like(x)
            K.conv_real(sp, x, y)
            K.device_status(sp)
            outs.append(y.cpu().numpy().astype(np.float64))
    rms = float(np.sqrt(np.mean(outs[1] ** 2)))
    d = np.abs(outs[0] - outs[1]) / rms
    top = np.argsort(d)[::-1][:8]
    print(json.dumps({"pixels": int(d.size), "rms": rms, "max_over_rms": float(d.max()),
                      "p99.99_over_rms": float(np.percentile(d, 99.99)),
                      "mean_over_rms": float(d.mean()),
                      "largest": [[int(p), float(d[p])] for p in top]}, indent=1))


if __name__ == "__main__":
    main()
