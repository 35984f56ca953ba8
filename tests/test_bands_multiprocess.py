"""Latitude-band decomposition across ranks, world size 2 over gloo on CPU.

Each rank computes only its band of output rings (here with the FP64 oracle,
standing in for ksconv.conv_real_rings on a GPU), the bands are gathered, and
the assembled map must equal the whole-map result exactly.  Also checks the
max-over-ranks timing reduction used by the benchmark."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1409_4441_gb300 import bands, inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nside, tc, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        c = inputs.gaussian_beam(3 * nside - 1, np.radians(8.0))
        m = inputs.white_noise_map(nside, 3)
        bl = bands.ring_bands(nside, world)
        lo, hi = bl[rank]
        s, e = bands.band_pixels(nside, lo, hi)
        out = torch.zeros(12 * nside * nside, dtype=torch.float64)
        if e > s:
            part, _ = O.brute_conv(nside, m, tc, c=c, out_pix=np.arange(s, e))
            out[s:e] = torch.from_numpy(part)
        bands.gather_bands(out, nside, bl)
        t = bands.max_over_ranks(1.0 + rank)
        q.put((rank, out.numpy().copy(), t))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_band_gather_equals_whole_map(world):
    import oracle as O
    nside, tc = 8, np.radians(20.0)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nside, tc, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    c = inputs.gaussian_beam(3 * nside - 1, np.radians(8.0))
    whole, _ = O.brute_conv(nside, inputs.white_noise_map(nside, 3), tc, c=c)
    for rank, out, t in res:
        assert np.array_equal(out, whole)
        assert t == float(world)


def test_ring_bands_cover_and_balance():
    for nside in (1, 4, 64, 2048):
        for n in (1, 2, 3, 8):
            bl = bands.ring_bands(nside, n)
            assert bl[0][0] == 1 and bl[-1][1] == 4 * nside - 1
            for (a, b), (c, d) in zip(bl, bl[1:]):
                assert c == b + 1
            if nside >= 64:
                px = [np.diff(bands.band_pixels(nside, lo, hi))[0] for lo, hi in bl]
                assert max(px) - min(px) <= 8 * nside  # boundaries fall on rings: <= 2 rings
    s, e = bands.band_pixels(4, 1, 15)
    assert (s, e) == (0, 12 * 16)
