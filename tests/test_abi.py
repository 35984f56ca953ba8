"""The C ABI library loads and exports every symbol include/ksconv.h declares;
host-side argument validation (no device work, no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def K():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1409_4441_gb300 import ksconv
    return ksconv


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ksconv.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ksc_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(K):
    syms = declared_symbols()
    assert len(syms) >= 17
    lib = ctypes.CDLL(K.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in ksconv.h but not exported"
    assert sorted(K.EXPORTS) == syms


def test_status_strings_and_defaults(K):
    assert K._lib.ksc_status_string(K.KSC_ERR_ARG) == b"KSC_ERR_ARG"
    assert K._lib.ksc_status_string(-99) == b"KSC_ERR_UNKNOWN"
    o = K.default_opts()
    assert (o.mode, o.oversample, o.svd_rcond, o.alpha, o.n_intervals, o.path, o.tensor) == \
        (0, 2, 1e-6, 5.0, 0, 0, 0)


@pytest.mark.parametrize("nside,lcut,tc,lmax", [
    (3, 10, 0.1, 40),      # nside not a power of two
    (16384, 10, 0.1, 40),  # nside too large
    (16, 40, 0.1, 40),     # l_cut >= lmax
    (16, 10, 0.0, 40),     # theta_cut <= 0
    (16, 10, 4.0, 40),     # theta_cut > pi
    (16, 10, 0.1, 0),      # lmax < 1
])
def test_invalid_arguments_are_rejected_before_device_work(K, nside, lcut, tc, lmax):
    b = np.ones(max(lmax, 0) + 1)
    with pytest.raises(K.KsconvError) as ei:
        K.make_split(b, nside, lcut, tc)
    assert ei.value.code == K.KSC_ERR_ARG


def test_null_pointers_rejected(K):
    lib = K._lib
    assert lib.ksc_conv_real(None, None, None, None) == K.KSC_ERR_ARG
    assert lib.ksc_split_info(None, None) == K.KSC_ERR_ARG
    assert lib.ksc_make_split(None, 10, 4, 2, 0.1, None, None, None) == K.KSC_ERR_ARG
    lib.ksc_free_split(None)  # no-op


def test_sht_arguments_rejected_before_device_work(K):
    lib = K._lib
    for nside, lmax in ((3, 8), (16, 65), (16, -1), (16384, 8)):
        assert lib.ksc_sht_map2alm(nside, lmax, 16, 16, None) == K.KSC_ERR_ARG
        assert lib.ksc_sht_alm2map(nside, lmax, 16, 16, None) == K.KSC_ERR_ARG
    assert lib.ksc_sht_map2alm(16, 32, None, 16, None) == K.KSC_ERR_ARG
    assert lib.ksc_conv_harmonic(None, 16, 16, 0, None) == K.KSC_ERR_ARG
