"""Rounding error of the belt kernel's summation order, emulated on the host (no GPU):

    python tests/belt_rounding.py [--rings 600] [--procs 6]

Belt x belt ring pairs of the nside-2048 benchmark split (l_max 4096, 5' Gaussian beam,
l_cut 1024, theta_cut 240'), the benchmark's white-noise map.  The weights are the oracle's
cubic Hermite interpolant of K_r at the exact chord, rounded to FP32.  Every FMA is emulated
as the FP64 sum of the exact product and the FP32 accumulator, rounded to FP32.  Each
output pixel of a ring is summed in the belt kernel's order:

  - per input ring, a window of Delta from d0 = -w to w (zero weight outside the cut),
    padded to blocks of 26 steps;
  - each block accumulates into a fresh FP32 partial, which is added into the ring pair's
    partial;
  - the ring pair's partial folds into the Kahan-compensated total.

Two fold policies are compared against the FP64 sum of the same products (the final
multiply by 4 pi / Npix included):

  per_pair  one fold at the end of each ring pair;
  peak      also a fold right after the half block (13 steps) holding Delta = 3, in ring
            pairs whose closest approach is within an eighth of the cut (the kernel's).

Prints, per policy, the maximum, the 99.99th and 99.999th percentiles and the count above
1e-6 of each ring's output rms.  This is an emulation of the order of operations, not a
run of the kernel; no test reads it.  About 10 minutes on 6 cores for 600 rings.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1409_4441_gb300 import inputs  # noqa: E402

ARC = inputs.ARCMIN
NSIDE, LMAX, FWHM, LCUT, TC = 2048, 4096, 5.0 * ARC, 1024, 240.0 * ARC
N_INT = 4371     # table intervals of the benchmark split
BLOCK, HALF = 26, 13
POLICIES = ("per_pair", "peak")

_S = {}


def _setup():
    c = inputs.gaussian_beam(LMAX, FWHM)
    c[: LCUT + 1] = 0.0
    _S["tab"] = O.hermite_nodes(c, TC, N_INT)
    _S["rings"] = O.ring_table(NSIDE)
    _S["map"] = inputs.white_noise_map(NSIDE, inputs.seed_for(3)).astype(np.float32)


def _kahan(s, c, v):
    f32 = np.float32
    y = f32(v - c)
    t = f32(s + y)
    return t, f32(f32(t - s) - y)


def _ring(i):
    """Errors / output rms of every pixel of belt ring i under each policy."""
    if not _S:
        _setup()
    f32, f64 = np.float32, np.float64
    z, s, _, st, ph = _S["rings"]
    m = _S["map"]
    tabK, tabD = _S["tab"]
    L = 4 * NSIDE
    dc = O.chord_cut(TC)
    zi, si, phi = z[i - 1], s[i - 1], ph[i - 1]
    ref = np.zeros(L)
    tot = {p: [np.zeros(L, f32), np.zeros(L, f32)] for p in POLICIES}
    Ds = np.arange(-(L // 2), L // 2)
    for q in range(NSIDE, 3 * NSIDE + 1):
        zq, sq, phq = z[q - 1], s[q - 1], ph[q - 1]
        A = (zi - zq) ** 2 + (si - sq) ** 2
        if A > dc * dc:
            continue
        d2 = A + 4 * si * sq * np.sin((phq - phi + Ds * 2 * np.pi / L) / 2) ** 2
        inside = d2 <= dc * dc
        if not inside.any():
            continue
        w_half = int(np.abs(Ds[inside]).max())
        d0 = -w_half
        nd = -(-(2 * w_half + 1) // BLOCK) * BLOCK
        D = d0 + np.arange(nd)
        dd = d2[np.clip(D + L // 2, 0, L - 1)]
        ok = (D >= -(L // 2)) & (D < L // 2) & (dd <= dc * dc)
        w = np.zeros(nd, f32)
        w[ok] = f32(O.hermite_eval(tabK, tabD, TC, np.sqrt(dd[ok])))
        x = m[st[q - 1]: st[q - 1] + L]
        base = (np.arange(L) + d0) % L
        near = A < (dc / 8) ** 2
        jfold = ((3 - d0) // HALF + 1) * HALF - 1 if near else -1
        acc = {p: np.zeros(L, f32) for p in POLICIES}
        ring = {p: np.zeros(L, f32) for p in POLICIES}
        for j in range(nd):
            if w[j] == 0.0:
                pr = None
            else:
                pr = f64(w[j]) * f64(x[(base + j) % L])
                ref += pr
            for p in POLICIES:
                if pr is not None:
                    acc[p] = f32(pr + f64(acc[p]))
                end = (j + 1) % BLOCK == 0
                mid = p == "peak" and j == jfold
                if end or mid:
                    ring[p] = f32(ring[p] + acc[p])
                    acc[p][:] = 0
                if mid:
                    tot[p] = list(_kahan(tot[p][0], tot[p][1], ring[p]))
                    ring[p][:] = 0
        for p in POLICIES:
            tot[p] = list(_kahan(tot[p][0], tot[p][1], ring[p]))
    dom = 4 * np.pi / (12 * NSIDE * NSIDE)
    refo = ref * dom
    rms = np.sqrt(np.mean(refo ** 2))
    return {p: np.abs(f64(f32(tot[p][0] * f32(dom))) - refo) / rms for p in POLICIES}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rings", type=int, default=600)
    ap.add_argument("--procs", type=int, default=6)
    a = ap.parse_args()
    step = max(1, (2 * NSIDE - 2) // a.rings)
    rings = [NSIDE + 13 + k * step for k in range(a.rings)]
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = pool.map(_ring, rings)
    out = {"rings": len(rings), "pixels": len(rings) * 4 * NSIDE}
    for p in POLICIES:
        e = np.concatenate([r[p] for r in res])
        out[p] = {"max": float(e.max()), "p99.99": float(np.percentile(e, 99.99)),
                  "p99.999": float(np.percentile(e, 99.999)), "above_1e-6": int((e > 1e-6).sum())}
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
