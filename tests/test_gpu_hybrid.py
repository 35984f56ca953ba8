"""The concurrent split convolution of Fig. 1: the real-space half runs asynchronously on the
GPU (ksc_conv_real returns at once) while the host computes the harmonic half (here the
oracle's FP64 spherical-harmonic transform stands in for the caller's SHT library); the sum
of the two halves is the split convolution, and the wall time is about the larger of the two
halves, not their sum."""
import time

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
    return ksconv


def test_gpu_and_host_halves_overlap(K):
    nside, lmax, lcut, fwhm, tc = 512, 1024, 256, 20 * ARC, 960 * ARC
    b = inputs.gaussian_beam(lmax, fwhm)
    cl = inputs.cl_grf(lmax)
    alm0 = inputs.grf_alm(lmax, cl, inputs.seed_for(2))
    m = O.alm2map(nside, alm0, lmax).astype(np.float32)
    m64 = m.astype(np.float64)
    with K.make_split(b, nside, lcut, tc, cl_in=cl) as sp:
        kh = K.split_harmonic(sp)
        x = torch.tensor(m, device="cuda")
        y = torch.empty_like(x)
        kf = np.zeros(lmax + 1)
        kf[: lcut + 1] = kh
        stream = torch.cuda.Stream()
        # each half alone
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(12):
                K.conv_real(sp, x, y, stream=stream)
        stream.synchronize()
        t_gpu = time.perf_counter() - t0
        t0 = time.perf_counter()
        harm = O.sht_conv(nside, m64, kf)
        t_cpu = time.perf_counter() - t0
        # both at once: launch the GPU half, compute the harmonic half meanwhile
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(12):
                K.conv_real(sp, x, y, stream=stream)
        harm2 = O.sht_conv(nside, m64, kf)
        stream.synchronize()
        t_both = time.perf_counter() - t0
        K.device_status(sp, stream=stream)
        real = y.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(harm, harm2)
    ell = np.concatenate([np.arange(mm, lmax + 1) for mm in range(lmax + 1)])
    alm = O.map2alm(nside, m64, lmax)
    full = O.alm2map(nside, alm * b[ell], lmax)
    split = harm + real
    cs = O.alm2cl(O.map2alm(nside, split, lmax), lmax)
    cf = O.alm2cl(O.map2alm(nside, full, lmax), lmax)
    eps = O.eps_cl(cs, cf, lmin=2)
    print(f"\nGPU half {t_gpu * 1e3:.0f} ms, host half {t_cpu * 1e3:.0f} ms, concurrent "
          f"{t_both * 1e3:.0f} ms (sum {1e3 * (t_gpu + t_cpu):.0f}); eps_C {eps:.2e}")
    assert t_both < 0.9 * (t_gpu + t_cpu)
    assert eps < 1e-4
