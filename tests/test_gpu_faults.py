"""Failure handling without a GPU fault: host-side fault injection.

KSC_FAULT = "alloc:N" makes the N-th device allocation of a split construction (or of
the host path's first call) fail as an out-of-memory would.  Every such failure must
come back as KSC_ERR_NOMEM with a message, release what the construction had already
allocated (device memory in use afterwards equals device memory in use before), and
leave the library usable: the next construction without the fault convolves a map
within the oracle parity tolerance.
"""
import os

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
    assert torch.cuda.is_available()
    return ksconv


def _used():
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    return total - free


@pytest.mark.parametrize("n", [1, 2, 5, 9, 13, 14])
def test_allocation_fault_is_clean(K, n, monkeypatch):
    nside, tc = 16, np.radians(20.0)
    c = inputs.gaussian_beam(47, np.radians(6.0))
    torch.cuda.init()
    before = _used()
    monkeypatch.setenv("KSC_FAULT", f"alloc:{n}")
    with pytest.raises(K.KsconvError) as e:
        K.make_split_real(c, nside, tc)
    monkeypatch.delenv("KSC_FAULT")
    assert e.value.code == K.KSC_ERR_NOMEM
    assert _used() == before
    # the library is still usable
    m = inputs.white_noise_map(nside, 5).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        n_int = K.split_info(sp)["n_intervals"]
        x = torch.tensor(m, device="cuda")
        y = torch.empty_like(x)
        K.conv_real(sp, x, y)
        K.device_status(sp)
        got = y.cpu().numpy().astype(np.float64)
    ref, amb = O.brute_conv(nside, m.astype(np.float64), tc, table=O.hermite_nodes(c, tc, n_int))
    assert (np.abs(got - ref) <= 1e-6 * np.sqrt(np.mean(ref ** 2)) + amb).all()


def test_host_path_allocation_fault_is_clean(K, monkeypatch):
    nside, tc = 16, np.radians(20.0)
    c = inputs.gaussian_beam(47, np.radians(6.0))
    m = inputs.white_noise_map(nside, 6).astype(np.float32)
    with K.make_split_real(c, nside, tc) as sp:
        before = _used()
        monkeypatch.setenv("KSC_FAULT", "alloc:1")
        with pytest.raises(K.KsconvError) as e:
            K.conv_real_host(sp, m)
        monkeypatch.delenv("KSC_FAULT")
        assert e.value.code == K.KSC_ERR_NOMEM
        assert _used() == before
        out = K.conv_real_host(sp, m)  # now allocates its buffers and runs
        assert np.isfinite(out).all()
