"""The allocation-free table build (ksc_build_table_noalloc).

Some callers cannot allocate device memory where they need a table (a caching
allocator or fixed budget owns the device, a real-time loop cannot take
cudaMalloc's synchronisation, or the work is being captured into a CUDA
graph).  This entry point keeps its scratch in a built-in device array; here
it is checked, through the C ABI, against the allocating path
(ksc_make_split_real + ksc_split_table) on two calls in a row with different
kernels, so that the second call also shows the shared scratch carries no
state over from the first.  This file sorts last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1409_4441_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ARC = inputs.ARCMIN


@pytest.fixture(scope="module")
def K():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_4441_gb300 import ksconv
    assert torch.cuda.is_available()
    return ksconv


def _reference_table(K, c, nside, tc, n_int):
    with K.make_split_real(c, nside, tc, n_intervals=n_int) as sp:
        return K.split_table(sp)


def test_noalloc_table_matches_allocating_path(K):
    cases = []
    c1 = inputs.gaussian_beam(1535, 20 * ARC)
    c1[:257] = 0.0
    cases.append((c1, 512, 90 * ARC, 2101))
    c2 = inputs.gaussian_beam(4096, 5 * ARC)
    cases.append((c2, 2048, 240 * ARC, 8192))  # the largest table the scratch holds
    for c, nside, tc, n_int in cases:  # two calls in a row
        ref = _reference_table(K, c, nside, tc, n_int)
        d_c = torch.tensor(c, dtype=torch.float64, device="cuda")
        d_tab = torch.full((n_int, 4), float("nan"), dtype=torch.float32, device="cuda")
        K.build_table_noalloc(d_c, c.size - 1, tc, n_int, d_tab)
        torch.cuda.synchronize()
        got = d_tab.cpu().numpy()
        peak = np.abs(ref[:, 0]).max()
        np.testing.assert_allclose(got, ref, rtol=0, atol=2e-7 * peak)
        assert np.array_equal(got, ref)  # same kernels and inputs: identical bits


def test_noalloc_rejects_oversize_table(K):
    c = torch.ones(11, dtype=torch.float64, device="cuda")
    d_tab = torch.empty((8193, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(K.KsconvError) as ei:
        K.build_table_noalloc(c, 10, 0.1, 8193, d_tab)
    assert ei.value.code == K.KSC_ERR_ARG
    assert "8192" in str(ei.value)
