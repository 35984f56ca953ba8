"""Latitude-band decomposition of one map across ranks (Sec. 4: latitude bands
with theta_cut overlap).

Each rank holds the whole input map (it is at most a few hundred MB), convolves
the output rings of its band with ``ksconv.conv_real_rings`` and the bands are
then gathered.  Helpers here are host-side only: the partition of rings into
contiguous bands of balanced work, the pixel range of a band, and the gather
of band outputs through ``torch.distributed`` (any backend).
"""
from __future__ import annotations

import numpy as np


def ring_lengths(nside: int) -> np.ndarray:
    """Pixels per HEALPix ring, rings 1..4 nside - 1."""
    i = np.arange(1, 4 * nside)
    return np.where(i < nside, 4 * i, np.where(i <= 3 * nside, 4 * nside, 4 * (4 * nside - i)))


def ring_bands(nside: int, n_parts: int, work=None):
    """Split rings 1..4 nside - 1 into n_parts contiguous bands of about equal
    work (default: pixels per ring, i.e. output pixels; the in-disc pair count
    per output pixel is nearly uniform).  Returns [(ring_lo, ring_hi), ...]
    (1-based, inclusive); a band may be empty (lo > hi) when n_parts exceeds
    the number of rings."""
    w = ring_lengths(nside).astype(np.float64) if work is None else np.asarray(work, float)
    nr = w.size
    cum = np.concatenate([[0.0], np.cumsum(w)])
    bounds = [0]
    for p in range(1, n_parts):
        target = cum[-1] * p / n_parts
        bounds.append(int(np.clip(np.searchsorted(cum, target), bounds[-1], nr)))
    bounds.append(nr)
    return [(bounds[p] + 1, bounds[p + 1]) for p in range(n_parts)]


def band_pixels(nside: int, ring_lo: int, ring_hi: int):
    """[start, end) pixel offsets (RING order) of rings ring_lo..ring_hi."""
    ln = ring_lengths(nside)
    start = int(ln[: ring_lo - 1].sum())
    end = int(ln[:ring_hi].sum()) if ring_hi >= ring_lo else start
    return start, end


def gather_bands(full_out, nside: int, bands, group=None):
    """Assemble the full output on every rank: rank p owns band p of full_out
    (a 1-D torch tensor of 12 nside^2 values); the other entries are filled in
    from the owners with all_gather of equal-length padded slices."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    spans = [band_pixels(nside, lo, hi) for lo, hi in bands]
    width = max(e - s for s, e in spans)
    mine = torch.zeros(width, dtype=full_out.dtype, device=full_out.device)
    s, e = spans[rank]
    mine[: e - s] = full_out[s:e]
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    for p, (s, e) in enumerate(spans):
        full_out[s:e] = parts[p][: e - s]
    return full_out


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (the benchmark's timing rule)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
