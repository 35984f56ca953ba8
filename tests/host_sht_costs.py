"""Time the harmonic half of the split convolution on the host (run on the host of the machine with the GPU):

    python tests/host_sht_costs.py [--out tests/golden/host_sht_times.csv]

The paper's CPU half (Fig. 1) is an SHT pair up to l_cut: analysis of the map, the kernel
applied to a_lm, synthesis.  Here it is the oracle's ring SHT (FFT along rings, Legendre
recurrence in l; OpenMP over the host's cores), timed at several (nside, l_cut) with l_max =
2 nside, so that the host cost model of Eq. 8 (t = h0 + h1 l_cut^2 l_max / 4096^3) can be
refitted to this host (tests/test_scan.py).  Wall-clock seconds, best of two.
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

CASES = [(256, 64), (256, 128), (256, 256), (512, 128), (512, 256), (512, 512),
         (1024, 256), (1024, 512), (1024, 1024)]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "host_sht_times.csv"))
    args = ap.parse_args()
    O.build()
    rows = []
    for nside, lcut in CASES:
        m = inputs.white_noise_map(nside, inputs.seed_for(6, nside))
        k = inputs.gaussian_beam(lcut, np.radians(1.0))
        ell = np.concatenate([np.arange(mm, lcut + 1) for mm in range(lcut + 1)])
        best = np.inf
        for _ in range(2):
            t0 = time.perf_counter()
            alm = O.map2alm(nside, m, lcut)
            O.alm2map(nside, alm * k[ell], lcut)
            best = min(best, time.perf_counter() - t0)
        rows.append((nside, 2 * nside, lcut, 1e3 * best))
        print(f"nside {nside} l_cut {lcut}: {1e3 * best:.1f} ms", flush=True)
    with open(args.out, "w") as f:
        f.write("# Host time of the harmonic half (oracle ring SHT: analysis to l_cut, kernel\n")
        f.write(f"# applied, synthesis), written by tests/host_sht_costs.py on {os.cpu_count()} "
                "host cores\n")
        f.write("# of the machine with the GPU; l_max = 2 nside (the map's band limit in Eq. 8's form).\n")
        f.write("nside,lmax,l_cut,t_ms\n")
        for r in rows:
            f.write(f"{r[0]},{r[1]},{r[2]},{r[3]:.3f}\n")


if __name__ == "__main__":
    main()
