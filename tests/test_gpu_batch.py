"""Batched persistent launches, CUDA-graph replay and the tile autotuner (ksc_batch_*).

A batch merges the work items of many (split, map) entries into one list per kernel and
tile variant and runs each list as one persistent launch.  Its kernels are separate
instantiations of the single-split kernels' per-item code, free to contract multiply-adds
differently, and the half-size gather tile regroups the FP32 partial sums: batch outputs
match single calls to FP32 rounding (1e-6 of the rms, the per-pixel tolerance), repeated
runs of one batch match bit for bit, and entries are checked against the FP64 oracle.
"""
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


# (nside, theta_cut deg, lmax, fwhm deg): ragged nside, beam and cut
SPECS = [(16, 12.0, 47, 4.0), (32, 6.0, 95, 2.5), (64, 4.0, 191, 1.5), (128, 2.0, 383, 0.8)]


def _entries(K, n_rep=2):
    sps = [K.make_split_real(inputs.gaussian_beam(lm, np.radians(fw)), ns, np.radians(td))
           for ns, td, lm, fw in SPECS]
    splits, ins = [], []
    for i, sp in enumerate(sps):
        ns = SPECS[i][0]
        for r in range(n_rep):  # repeated splits: a small map stack per kernel
            splits.append(sp)
            m = inputs.white_noise_map(ns, 1000 + 10 * i + r).astype(np.float32)
            ins.append(torch.tensor(m, device="cuda"))
    return sps, splits, ins


def _close(a, r, rel=1e-6):
    a, r = a.cpu().numpy().astype(np.float64), r.cpu().numpy().astype(np.float64)
    rms = np.sqrt(np.mean(r ** 2))
    assert not np.isnan(a).any()
    assert np.abs(a - r).max() <= rel * rms, np.abs(a - r).max() / rms


def _singles(K, splits, ins):
    outs = []
    for sp, x in zip(splits, ins):
        y = torch.empty_like(x)
        K.conv_real(sp, x, y)
        outs.append(y)
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_single_calls_and_replays_bitwise(K, use_graph):
    sps, splits, ins = _entries(K)
    ref = _singles(K, splits, ins)
    with K.Batch(splits, use_graph=use_graph) as b:
        info = b.info()
        assert info["n_entries"] == len(splits) and info["n_splits"] == len(SPECS)
        # one persistent launch per kernel and tile variant in use
        assert info["n_launches"] <= 4
        outs = [torch.full_like(x, float("nan")) for x in ins]
        b.run(ins, outs)
        b.status()
        for a, r in zip(outs, ref):
            _close(a, r)
        # replay with fresh output buffers (the pointer table is re-uploaded), twice
        for _ in range(2):
            outs2 = [torch.full_like(x, float("nan")) for x in ins]
            b.run(ins, outs2)
            torch.cuda.synchronize()
            for a, r in zip(outs2, outs):
                assert torch.equal(a, r)
    for s in sps:
        s.close()


def test_autotune_then_parity(K):
    sps, splits, ins = _entries(K, n_rep=1)
    ref = _singles(K, splits, ins)
    outs = [torch.empty_like(x) for x in ins]
    with K.Batch(splits) as b:
        rep = b.autotune(ins, outs)
        groups = rep["groups"]
        assert [g["nside"] for g in groups] == [s[0] for s in SPECS]
        for g in groups:
            assert g["belt_variant"] in (0, 1) and g["sym_variant"] in (0, 1, 2)
            assert min(g["ms_belt"]) > 0 and min(g["ms_sym"]) > 0
            # the choice is the faster of the two timings
            assert g["ms_belt"][g["belt_variant"]] == min(g["ms_belt"])
            assert g["ms_sym"][g["sym_variant"]] == min(g["ms_sym"])
        assert [(g["belt_variant"], g["sym_variant"]) for g in b.info()["groups"]] == \
            [(g["belt_variant"], g["sym_variant"]) for g in groups]
        b.run(ins, outs)
        b.status()
        for a, r in zip(outs, ref):
            _close(a, r)
    # a new batch over the same splits starts from the cached choice
    with K.Batch(splits) as b2:
        assert [(g["belt_variant"], g["sym_variant"]) for g in b2.info()["groups"]] == \
            [(g["belt_variant"], g["sym_variant"]) for g in groups]
    # one entry of the tuned batch against the FP64 oracle (tabulated kernel)
    ns, td, lm, fw = SPECS[2]
    c = inputs.gaussian_beam(lm, np.radians(fw))
    n_int = K.split_info(sps[2])["n_intervals"]
    m = ins[2].cpu().numpy().astype(np.float64)
    orc, amb = O.brute_conv(ns, m, np.radians(td), table=O.hermite_nodes(c, np.radians(td), n_int))
    got = outs[2].cpu().numpy().astype(np.float64)
    rms = np.sqrt(np.mean(orc ** 2))
    assert np.all(np.abs(got - orc) <= 1e-6 * rms + amb)
    for s in sps:
        s.close()


def test_batch_mixed_with_general_path_split(K):
    """A split on the general (reference) path rides along as its own launch."""
    ns, td, lm, fw = SPECS[1]
    c = inputs.gaussian_beam(lm, np.radians(fw))
    fast = K.make_split_real(c, ns, np.radians(td))
    gen = K.make_split_real(c, ns, np.radians(td), path=1)
    x = torch.tensor(inputs.white_noise_map(ns, 77).astype(np.float32), device="cuda")
    ref = _singles(K, [fast, gen], [x, x])
    for use_graph in (False, True):
        with K.Batch([fast, gen], use_graph=use_graph) as b:
            for _ in range(2):  # new output buffers each time
                outs = [torch.empty_like(x), torch.empty_like(x)]
                b.run([x, x], outs)
                torch.cuda.synchronize()
                _close(outs[0], ref[0])
                assert torch.equal(outs[1], ref[1])  # the same general-path launch
    fast.close()
    gen.close()


def test_batch_rejects_bad_pointers(K):
    ns, td, lm, fw = SPECS[0]
    with K.make_split_real(inputs.gaussian_beam(lm, np.radians(fw)), ns, np.radians(td)) as sp:
        x = torch.zeros(O.npix(ns), device="cuda")
        with K.Batch([sp]) as b:
            with pytest.raises(K.KsconvError) as e:
                b.run([x], [x])
            assert e.value.code == K.KSC_ERR_ARG
            big = torch.zeros(O.npix(ns) + 1, device="cuda")
            with pytest.raises(K.KsconvError) as e:
                b.run([x], [big[1:]])  # 4-byte offset: misaligned
            assert e.value.code == K.KSC_ERR_ARG
