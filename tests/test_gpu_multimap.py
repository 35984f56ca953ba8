"""Multi-map convolution: the tcgen05 tensor-core paths (cap ring pairs by default, belt
ring pairs too with tensor=2; TF32 x3, FP32 accumulate) against the per-map FFMA path
and the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1409_4441_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_4441_gb300 import ksconv
    return ksconv


@pytest.mark.parametrize("tensor", [0, 2])
@pytest.mark.parametrize("nside,n_maps,tc_deg,lmax,fwhm_deg", [
    (16, 16, 20.0, 47, 6.0),     # one padded group, every ring pair wide
    (32, 70, 8.0, 95, 3.0),      # ragged last map group
    (64, 64, 6.0, 191, 2.0),     # the 2-degree nside-64 kernel
])
def test_tensor_multimap_matches_ffma_and_oracle(K, nside, n_maps, tc_deg, lmax, fwhm_deg, tensor):
    tc = np.radians(tc_deg)
    c = inputs.gaussian_beam(lmax, np.radians(fwhm_deg))
    maps = np.stack([inputs.white_noise_map(nside, 500 + i) for i in range(n_maps)]).astype(np.float32)
    x = torch.tensor(maps, device="cuda")
    with K.make_split_real(c, nside, tc, tensor=tensor) as sp, \
            K.make_split_real(c, nside, tc, tensor=1) as sf:
        yt = torch.full_like(x, float("nan"))
        K.conv_real_multimap(sp, x, yt, n_maps)
        yf = torch.full_like(x, float("nan"))
        K.conv_real_multimap(sf, x, yf, n_maps)
        K.device_status(sp)
        K.device_status(sf)
        n_int = K.split_info(sp)["n_intervals"]
        # stages compose to the whole call
        ys = torch.empty_like(x)
        K.conv_real_multimap_stage(sp, x, ys, n_maps, 1)
        K.conv_real_multimap_stage(sp, x, ys, n_maps, 2)
        K.device_status(sp)
        assert torch.equal(ys, yt)
    yt = yt.cpu().numpy().astype(np.float64)
    yf = yf.cpu().numpy().astype(np.float64)
    assert not np.isnan(yt).any()
    rms = np.sqrt(np.mean(yf ** 2))
    d = np.abs(yt - yf).max() / rms
    print(f"\nnside {nside}, {n_maps} maps, tensor={tensor}: max |tensor - ffma| / rms = {d:.2e}")
    assert d <= 2e-6
    j = n_maps - 1
    ref, amb = O.brute_conv(nside, maps[j].astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int))
    rms_j = np.sqrt(np.mean(ref ** 2))
    assert np.all(np.abs(yt[j] - ref) <= 2e-6 * rms_j + amb)
