"""Thin ctypes binding of libksconv (include/ksconv.h): argument marshalling only.

Every computation runs inside the CUDA/C++ library.  If ``libksconv.so`` is
missing this module raises on import: there is no CPU fallback.  Device arrays
are torch CUDA tensors (float32, contiguous); streams default to torch's
current stream.  Angles are radians.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libksconv.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libksconv.so not built ({LIB_PATH}); run paper_1409_4441_gb300/build.py "
                      "or __graft_entry__.build() first")

_lib = ctypes.CDLL(LIB_PATH)

KSC_OK = 0
KSC_ERR_ARG = -1
KSC_ERR_NOMEM = -2
KSC_ERR_CUDA = -3
KSC_ERR_TIMEOUT = -4
KSC_ERR_DEVICE_BOUNDS = -5
KSC_ERR_SVD = -6
KSC_ERR_UNSUPPORTED = -7
KSC_ERR_TIMEOUT_UNDRAINED = -8
MODES = {"lsq": 0, "sharp": 1, "none": 2}
KSC_CUT_C1 = 0    # default: the real-space kernel's value and slope vanish at theta_cut
KSC_CUT_C0 = 1    # value only
KSC_CUT_FREE = 2  # unconstrained fit (K_r may jump at the cut)

# Every symbol include/ksconv.h declares.
EXPORTS = [
    "ksc_default_opts", "ksc_make_split", "ksc_make_split_real", "ksc_split_info",
    "ksc_split_harmonic", "ksc_split_real_coeffs", "ksc_split_model", "ksc_split_table",
    "ksc_conv_real", "ksc_conv_real_rings", "ksc_conv_real_multimap", "ksc_conv_real_batch",
    "ksc_conv_real_host", "ksc_conv_real_stage", "ksc_conv_real_multimap_stage",
    "ksc_count_pairs", "ksc_device_status", "ksc_dphi_table_params", "ksc_dphi_odd_params",
    "ksc_probe_wait_timeout",
    "ksc_free_split", "ksc_build_table_noalloc",
    "ksc_batch_default_opts", "ksc_batch_create", "ksc_batch_run", "ksc_batch_autotune",
    "ksc_batch_info", "ksc_batch_status", "ksc_batch_free",
    "ksc_mlp_n_params", "ksc_mlp_create", "ksc_mlp_set_norm", "ksc_mlp_get_params",
    "ksc_mlp_set_params", "ksc_mlp_predict", "ksc_mlp_grad", "ksc_mlp_train", "ksc_mlp_select",
    "ksc_mlp_free",
    "ksc_sht_alm2map", "ksc_sht_map2alm", "ksc_conv_harmonic",
    "ksc_cost_pairs", "ksc_cost_model_default", "ksc_cost_eval", "ksc_cost_fit_gpu",
    "ksc_cost_fit_host", "ksc_split_features", "ksc_scan_default_opts", "ksc_scan_split",
    "ksc_status_string", "ksc_last_error",
]


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("oversample", ctypes.c_int),
                ("svd_rcond", ctypes.c_double), ("alpha", ctypes.c_double),
                ("n_intervals", ctypes.c_int), ("path", ctypes.c_int),
                ("tensor", ctypes.c_int), ("cut_continuity", ctypes.c_int),
                ("exact_weights", ctypes.c_int), ("cap_kernel", ctypes.c_int)]


class Desc(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("l_cut", ctypes.c_int), ("nside", ctypes.c_int),
                ("mode", ctypes.c_int), ("n_intervals", ctypes.c_int),
                ("n_unknowns", ctypes.c_int), ("n_kept", ctypes.c_int),
                ("theta_cut", ctypes.c_double), ("chord_cut", ctypes.c_double),
                ("sigma_rms", ctypes.c_double), ("frac_error", ctypes.c_double),
                ("n_pairs", ctypes.c_longlong), ("n_pairs_belt", ctypes.c_longlong),
                ("path", ctypes.c_int), ("frac_tabulated", ctypes.c_double)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int), ("per_sm_cap", ctypes.c_int)]


class TuneReport(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int), ("nside", ctypes.c_int * 8),
                ("belt_variant", ctypes.c_int * 8), ("sym_variant", ctypes.c_int * 8),
                ("ms_belt", (ctypes.c_double * 2) * 8), ("ms_sym", (ctypes.c_double * 3) * 8)]


class BatchDesc(ctypes.Structure):
    _fields_ = [("n_entries", ctypes.c_int), ("n_splits", ctypes.c_int),
                ("n_groups", ctypes.c_int), ("n_items_belt", ctypes.c_int),
                ("n_items_sym", ctypes.c_int), ("n_launches", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("n_pairs", ctypes.c_longlong),
                ("group_nside", ctypes.c_int * 8), ("group_belt_variant", ctypes.c_int * 8),
                ("group_sym_variant", ctypes.c_int * 8)]


class CostModel(ctypes.Structure):
    _fields_ = [("gpu_ms0", ctypes.c_double), ("gpu_ms_per_tpair", ctypes.c_double),
                ("host_ms0", ctypes.c_double), ("host_ms_eq8", ctypes.c_double),
                ("gpu_ms_per_tpair_ring", ctypes.c_double)]


class ScanOpts(ctypes.Structure):
    _fields_ = [("theta_lo", ctypes.c_double), ("theta_hi", ctypes.c_double),
                ("theta_step", ctypes.c_double), ("bound", ctypes.c_double),
                ("l_cut_fixed", ctypes.c_int), ("linear_steps", ctypes.c_int)]


class ScanRow(ctypes.Structure):
    _fields_ = [("theta_cut", ctypes.c_double), ("l_cut", ctypes.c_int),
                ("error", ctypes.c_double), ("t_gpu_ms", ctypes.c_double),
                ("t_host_ms", ctypes.c_double)]


_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_sig = {
    "ksc_default_opts": [ctypes.POINTER(Opts)],
    "ksc_make_split": [_vp, _i, _i, _i, _d, _vp, ctypes.POINTER(Opts), ctypes.POINTER(_vp)],
    "ksc_make_split_real": [_vp, _i, _i, _d, ctypes.POINTER(Opts), ctypes.POINTER(_vp)],
    "ksc_split_info": [_vp, ctypes.POINTER(Desc)],
    "ksc_split_harmonic": [_vp, _vp],
    "ksc_split_real_coeffs": [_vp, _vp],
    "ksc_split_model": [_vp, _vp],
    "ksc_split_table": [_vp, _vp],
    "ksc_conv_real": [_vp, _vp, _vp, _vp],
    "ksc_conv_real_rings": [_vp, _vp, _vp, _i, _i, _vp],
    "ksc_conv_real_multimap": [_vp, _vp, _vp, _i, _vp],
    "ksc_conv_real_batch": [_vp, _vp, _vp, _i, _vp],
    "ksc_conv_real_host": [_vp, _vp, _vp],
    "ksc_conv_real_stage": [_vp, _vp, _vp, _i, _vp],
    "ksc_conv_real_multimap_stage": [_vp, _vp, _vp, _i, _i, _vp],
    "ksc_count_pairs": [_vp, ctypes.POINTER(ctypes.c_longlong)],
    "ksc_dphi_table_params": [_d, _d, _d, _i, _d, _i, _d, _vp],
    "ksc_dphi_odd_params": [_d, _d, _d, _i, _d, _i, _d, _i, _vp],
    "ksc_probe_wait_timeout": [_vp, ctypes.c_int, _vp],
    "ksc_device_status": [_vp, _vp],
    "ksc_free_split": [_vp],
    "ksc_build_table_noalloc": [_vp, _i, _d, _i, _vp, _vp],
    "ksc_batch_default_opts": [ctypes.POINTER(BatchOpts)],
    "ksc_batch_create": [_vp, _i, ctypes.POINTER(BatchOpts), ctypes.POINTER(_vp)],
    "ksc_batch_run": [_vp, _vp, _vp, _vp],
    "ksc_batch_autotune": [_vp, _vp, _vp, _vp, ctypes.POINTER(TuneReport)],
    "ksc_batch_info": [_vp, ctypes.POINTER(BatchDesc)],
    "ksc_batch_status": [_vp, _vp],
    "ksc_batch_free": [_vp],
    "ksc_mlp_n_params": [],
    "ksc_mlp_create": [ctypes.c_ulonglong, ctypes.POINTER(_vp)],
    "ksc_mlp_set_norm": [_vp, _vp, _vp, _vp, _vp],
    "ksc_mlp_get_params": [_vp, _vp],
    "ksc_mlp_set_params": [_vp, _vp],
    "ksc_mlp_predict": [_vp, _vp, _i, _vp, _vp],
    "ksc_mlp_grad": [_vp, _vp, _vp, _i, _vp, _vp],
    "ksc_mlp_train": [_vp, _vp, _vp, _i, _i, ctypes.c_float, _vp, _vp],
    "ksc_mlp_select": [_vp, _vp, _i, _d, _d, _vp, ctypes.POINTER(_i), _vp],
    "ksc_mlp_free": [_vp],
    "ksc_sht_alm2map": [_i, _i, _vp, _vp, _vp],
    "ksc_sht_map2alm": [_i, _i, _vp, _vp, _vp],
    "ksc_conv_harmonic": [_vp, _vp, _vp, _i, _vp],
    "ksc_cost_model_default": [ctypes.POINTER(CostModel)],
    "ksc_cost_eval": [ctypes.POINTER(CostModel), _i, _i, _i, _d, _vp, _vp],
    "ksc_cost_fit_gpu": [_vp, _vp, _vp, _i, ctypes.POINTER(CostModel)],
    "ksc_cost_fit_host": [_vp, _vp, _vp, _i, ctypes.POINTER(CostModel)],
    "ksc_split_features": [_i, _vp, _vp, _vp, _vp, _vp],
    "ksc_scan_default_opts": [ctypes.POINTER(ScanOpts)],
    "ksc_scan_split": [_vp, _i, _i, _vp, ctypes.POINTER(ScanOpts), ctypes.POINTER(CostModel),
                       ctypes.POINTER(Opts), _vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)],
    "ksc_status_string": [_i],
    "ksc_last_error": [],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _i
_lib.ksc_free_split.restype = None
_lib.ksc_cost_pairs.argtypes = [_i, _d]
_lib.ksc_cost_pairs.restype = _d
_lib.ksc_batch_free.restype = None
_lib.ksc_mlp_free.restype = None
_lib.ksc_status_string.restype = ctypes.c_char_p
_lib.ksc_last_error.restype = ctypes.c_char_p


class KsconvError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.ksc_last_error().decode()
        super().__init__(f"{where}: {_lib.ksc_status_string(code).decode()} ({msg})")


def _check(rc: int, where: str):
    if rc != KSC_OK:
        raise KsconvError(rc, where)


def _dptr(t):
    """Device address of a torch CUDA tensor (float32, contiguous) or an int."""
    if isinstance(t, int):
        return t
    import torch
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


def _dptr_typed(t, dtype_name: str):
    """Device address of a contiguous CUDA tensor of the given dtype."""
    import torch
    if not t.is_cuda or t.dtype != getattr(torch, dtype_name) or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype_name} CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def default_opts(**kw) -> Opts:
    o = Opts()
    _check(_lib.ksc_default_opts(ctypes.byref(o)), "ksc_default_opts")
    names = {f for f, _ in Opts._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown split option {k!r} (known: {sorted(names)})")
        setattr(o, k, MODES[v] if k == "mode" else v)
    return o


class Split:
    """Owner of a ksc_split handle (freed on close/garbage collection)."""

    def __init__(self, handle: int):
        self._h = handle

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("split already freed")
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.ksc_free_split(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def make_split(b_l, nside: int, l_cut: int, theta_cut: float, cl_in=None, **opts) -> Split:
    """ksc_make_split: fit the Sec. 2 split of kernel b_l and build its device table."""
    b = np.ascontiguousarray(b_l, dtype=np.float64)
    cl = None if cl_in is None else np.ascontiguousarray(cl_in, dtype=np.float64)
    o = default_opts(**opts)
    h = _vp()
    _check(_lib.ksc_make_split(b.ctypes.data, b.size - 1, nside, l_cut, float(theta_cut),
                               None if cl is None else cl.ctypes.data, ctypes.byref(o),
                               ctypes.byref(h)), "ksc_make_split")
    return Split(h.value)


def make_split_real(c_l, nside: int, theta_cut: float, **opts) -> Split:
    """ksc_make_split_real: real-space part given by its Legendre coefficients."""
    c = np.ascontiguousarray(c_l, dtype=np.float64)
    o = default_opts(**opts)
    h = _vp()
    _check(_lib.ksc_make_split_real(c.ctypes.data, c.size - 1, nside, float(theta_cut),
                                    ctypes.byref(o), ctypes.byref(h)), "ksc_make_split_real")
    return Split(h.value)


def split_info(s: Split) -> dict:
    d = Desc()
    _check(_lib.ksc_split_info(s.handle, ctypes.byref(d)), "ksc_split_info")
    return {f: getattr(d, f) for f, _ in Desc._fields_}


def split_harmonic(s: Split) -> np.ndarray:
    info = split_info(s)
    out = np.zeros(max(info["l_cut"] + 1, 0))
    if out.size:
        _check(_lib.ksc_split_harmonic(s.handle, out.ctypes.data), "ksc_split_harmonic")
    return out


def split_real_coeffs(s: Split) -> np.ndarray:
    out = np.empty(split_info(s)["lmax"] + 1)
    _check(_lib.ksc_split_real_coeffs(s.handle, out.ctypes.data), "ksc_split_real_coeffs")
    return out


def split_model(s: Split) -> np.ndarray:
    out = np.empty(split_info(s)["lmax"] + 1)
    _check(_lib.ksc_split_model(s.handle, out.ctypes.data), "ksc_split_model")
    return out


def split_table(s: Split) -> np.ndarray:
    out = np.empty((split_info(s)["n_intervals"], 4), dtype=np.float32)
    _check(_lib.ksc_split_table(s.handle, out.ctypes.data), "ksc_split_table")
    return out


def count_pairs(s: Split) -> int:
    n = ctypes.c_longlong()
    _check(_lib.ksc_count_pairs(s.handle, ctypes.byref(n)), "ksc_count_pairs")
    return n.value


def dphi_table_params(A2: float, B2: float, c: float, n_int: int, hw: float, lq: int,
                      scale: float = 1.0) -> dict:
    """ksc_dphi_table_params: cell width (radians of x = dphi/2), cell count and the
    cut in |N| of one ring pair's dphi weight table (host only)."""
    out = np.zeros(3)
    _check(_lib.ksc_dphi_table_params(float(A2), float(B2), float(c), int(n_int), float(hw),
                                      int(lq), float(scale), out.ctypes.data),
           "ksc_dphi_table_params")
    return {"dx": float(out[0]), "ncell": int(out[1]), "ncut": float(out[2])}


def dphi_odd_params(A2: float, B2: float, c: float, n_int: int, hw: float, lq: int,
                    scale: float = 1.0, cap: int = 4096) -> dict:
    """ksc_dphi_odd_params: the lockstep gather's odd-step table of one ring pair
    (cell width in x = dphi/2, m, off, zero cell nct, ncut); host only."""
    out = np.zeros(5)
    _check(_lib.ksc_dphi_odd_params(float(A2), float(B2), float(c), int(n_int), float(hw),
                                    int(lq), float(scale), int(cap), out.ctypes.data),
           "ksc_dphi_odd_params")
    return {"width": out[0], "m": int(out[1]), "off": int(out[2]), "nct": int(out[3]),
            "ncut": int(out[4])}

def probe_wait_timeout(s: Split, max_polls: int = 0, stream=None):
    """Run the bounded-wait failure path once (max_polls <= 0: the kernels' limit)."""
    _check(_lib.ksc_probe_wait_timeout(s.handle, int(max_polls), _stream(stream)),
           "ksc_probe_wait_timeout")


def device_status(s: Split, stream=None):
    """Synchronize the stream and raise if a device-side check fired."""
    _check(_lib.ksc_device_status(s.handle, _stream(stream)), "ksc_device_status")


def conv_real(s: Split, d_in, d_out, stream=None):
    _check(_lib.ksc_conv_real(s.handle, _dptr(d_in), _dptr(d_out), _stream(stream)),
           "ksc_conv_real")
    return d_out


def conv_real_stage(s: Split, d_in, d_out, stage: int, stream=None):
    _check(_lib.ksc_conv_real_stage(s.handle, _dptr(d_in), _dptr(d_out), stage, _stream(stream)),
           "ksc_conv_real_stage")
    return d_out


def conv_real_multimap_stage(s: Split, d_in, d_out, n_maps: int, stage: int, stream=None):
    _check(_lib.ksc_conv_real_multimap_stage(s.handle, _dptr(d_in), _dptr(d_out), n_maps, stage,
                                             _stream(stream)), "ksc_conv_real_multimap_stage")
    return d_out


def conv_real_rings(s: Split, d_in, d_out, ring_lo: int, ring_hi: int, stream=None):
    _check(_lib.ksc_conv_real_rings(s.handle, _dptr(d_in), _dptr(d_out), ring_lo, ring_hi,
                                    _stream(stream)), "ksc_conv_real_rings")
    return d_out


def conv_real_multimap(s: Split, d_in, d_out, n_maps: int, stream=None):
    _check(_lib.ksc_conv_real_multimap(s.handle, _dptr(d_in), _dptr(d_out), n_maps,
                                       _stream(stream)), "ksc_conv_real_multimap")
    return d_out


def conv_real_batch(splits, d_ins, d_outs, stream=None):
    n = len(splits)
    hs = (_vp * n)(*[s.handle for s in splits])
    ins = (_vp * n)(*[_dptr(t) for t in d_ins])
    outs = (_vp * n)(*[_dptr(t) for t in d_outs])
    _check(_lib.ksc_conv_real_batch(hs, ins, outs, n, _stream(stream)), "ksc_conv_real_batch")
    return d_outs


def conv_real_host(s: Split, h_in, h_out=None):
    """Host float32 map in, host float32 map out (synchronous)."""
    if isinstance(h_in, np.ndarray):
        hi = np.ascontiguousarray(h_in, dtype=np.float32)
        ho = np.empty_like(hi) if h_out is None else h_out
        _check(_lib.ksc_conv_real_host(s.handle, hi.ctypes.data, ho.ctypes.data),
               "ksc_conv_real_host")
        return ho
    # pinned torch CPU tensors
    ho = h_out
    _check(_lib.ksc_conv_real_host(s.handle, h_in.data_ptr(), ho.data_ptr()),
           "ksc_conv_real_host")
    return ho


def build_table_noalloc(d_c, lmax: int, theta_cut: float, n_intervals: int, d_table,
                        stream=None):
    """ksc_build_table_noalloc: the K_r table from device coefficients d_c
    (float64, lmax+1) into d_table (float32, n_intervals x 4), without any
    device allocation (for callers that cannot allocate; see ksconv.h)."""
    _check(_lib.ksc_build_table_noalloc(_dptr_typed(d_c, "float64"), lmax, float(theta_cut),
                                        n_intervals, _dptr_typed(d_table, "float32"),
                                        _stream(stream)), "ksc_build_table_noalloc")
    return d_table


class Batch:
    """A ksc_batch: entries (split, map) run as persistent launches, optionally
    replayed as a CUDA graph.  Keeps its splits alive."""

    def __init__(self, splits, use_graph: bool = True, per_sm_cap: int = 0):
        self._splits = list(splits)
        n = len(self._splits)
        o = BatchOpts()
        _check(_lib.ksc_batch_default_opts(ctypes.byref(o)), "ksc_batch_default_opts")
        o.use_graph = 1 if use_graph else 0
        o.per_sm_cap = int(per_sm_cap)
        hs = (_vp * n)(*[s.handle for s in self._splits])
        h = _vp()
        _check(_lib.ksc_batch_create(hs, n, ctypes.byref(o), ctypes.byref(h)), "ksc_batch_create")
        self._h = h.value

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("batch already freed")
        return self._h

    def _ptrs(self, d_ins, d_outs):
        n = len(self._splits)
        if len(d_ins) != n or len(d_outs) != n:
            raise ValueError(f"expected {n} input and output maps")
        return (_vp * n)(*[_dptr(t) for t in d_ins]), (_vp * n)(*[_dptr(t) for t in d_outs])

    def run(self, d_ins, d_outs, stream=None):
        ins, outs = self._ptrs(d_ins, d_outs)
        _check(_lib.ksc_batch_run(self.handle, ins, outs, _stream(stream)), "ksc_batch_run")
        return d_outs

    def autotune(self, d_ins, d_outs, stream=None) -> dict:
        ins, outs = self._ptrs(d_ins, d_outs)
        r = TuneReport()
        _check(_lib.ksc_batch_autotune(self.handle, ins, outs, _stream(stream), ctypes.byref(r)),
               "ksc_batch_autotune")
        return {"groups": [{"nside": r.nside[g], "belt_variant": r.belt_variant[g],
                            "sym_variant": r.sym_variant[g],
                            "ms_belt": [r.ms_belt[g][0], r.ms_belt[g][1]],
                            "ms_sym": [r.ms_sym[g][v] for v in range(3)]}
                           for g in range(r.n_groups)]}

    def info(self) -> dict:
        d = BatchDesc()
        _check(_lib.ksc_batch_info(self.handle, ctypes.byref(d)), "ksc_batch_info")
        out = {f: getattr(d, f) for f, _ in BatchDesc._fields_ if not f.startswith("group_")}
        out["groups"] = [{"nside": d.group_nside[g], "belt_variant": d.group_belt_variant[g],
                          "sym_variant": d.group_sym_variant[g]} for g in range(min(d.n_groups, 8))]
        return out

    def status(self, stream=None):
        _check(_lib.ksc_batch_status(self.handle, _stream(stream)), "ksc_batch_status")

    def close(self):
        if getattr(self, "_h", None):
            _lib.ksc_batch_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _f32_host(a, cols):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != cols:
        raise ValueError(f"expected an (n, {cols}) array")
    return a


class MLP:
    """The surrogate split selector (ksc_mlp_*): a 4-64-64-2 network trained and
    evaluated by the library's CUDA kernels.  Device arrays are float32 CUDA
    tensors of shape (n, 4) inputs / (n, 2) targets."""

    def __init__(self, seed: int = 0):
        h = _vp()
        _check(_lib.ksc_mlp_create(ctypes.c_ulonglong(seed), ctypes.byref(h)), "ksc_mlp_create")
        self._h = h.value

    @staticmethod
    def n_params() -> int:
        return _lib.ksc_mlp_n_params()

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("model already freed")
        return self._h

    def set_norm(self, x_mean, x_std, y_mean, y_std):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (x_mean, x_std, y_mean, y_std)]
        _check(_lib.ksc_mlp_set_norm(self.handle, *[v.ctypes.data for v in a]), "ksc_mlp_set_norm")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params(), dtype=np.float32)
        _check(_lib.ksc_mlp_get_params(self.handle, out.ctypes.data), "ksc_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params():
            raise ValueError("wrong parameter count")
        _check(_lib.ksc_mlp_set_params(self.handle, p.ctypes.data), "ksc_mlp_set_params")

    def predict(self, d_x, d_y=None, stream=None):
        import torch
        n = d_x.shape[0]
        if d_y is None:
            d_y = torch.empty((n, 2), dtype=torch.float32, device=d_x.device)
        _check(_lib.ksc_mlp_predict(self.handle, _dptr(d_x), n, _dptr(d_y), _stream(stream)),
               "ksc_mlp_predict")
        return d_y

    def grad(self, d_x, d_t):
        g = np.empty(self.n_params(), dtype=np.float32)
        loss = ctypes.c_float()
        _check(_lib.ksc_mlp_grad(self.handle, _dptr(d_x), _dptr(d_t), d_x.shape[0], g.ctypes.data,
                                 ctypes.byref(loss)), "ksc_mlp_grad")
        return g, float(loss.value)

    def train(self, d_x, d_t, epochs: int, lr: float = 1e-3, stream=None) -> float:
        loss = ctypes.c_float()
        _check(_lib.ksc_mlp_train(self.handle, _dptr(d_x), _dptr(d_t), d_x.shape[0], int(epochs),
                                  ctypes.c_float(lr), _stream(stream), ctypes.byref(loss)),
               "ksc_mlp_train")
        return float(loss.value)

    def select(self, h_x, log10_bound: float, margin: float = 0.0, host_ms=None):
        """Index of the least-cost candidate whose predicted log10 eps_C clears the
        bound by `margin` decades (-1 if none), cost = max(predicted GPU ms,
        host_ms[i]) (host_ms None: GPU time only); and the (n, 2) predictions."""
        x = _f32_host(h_x, 4)
        pred = np.empty((x.shape[0], 2), dtype=np.float32)
        best = ctypes.c_int()
        hp = None
        if host_ms is not None:
            hm = np.ascontiguousarray(host_ms, dtype=np.float64)
            if hm.size != x.shape[0]:
                raise ValueError("host_ms needs one value per candidate")
            hp = hm.ctypes.data
        _check(_lib.ksc_mlp_select(self.handle, x.ctypes.data, x.shape[0], float(log10_bound),
                                   float(margin), hp, ctypes.byref(best), pred.ctypes.data),
               "ksc_mlp_select")
        return int(best.value), pred

    def close(self):
        if getattr(self, "_h", None):
            _lib.ksc_mlp_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _dptr_alm(t, lmax: int):
    """Device address of a contiguous complex128 CUDA tensor of n_alm(lmax) entries."""
    if isinstance(t, int):
        return t
    import torch
    if not t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous():
        raise ValueError("expected a contiguous complex128 CUDA tensor")
    if t.numel() != n_alm(lmax):
        raise ValueError(f"expected {n_alm(lmax)} a_lm, got {t.numel()}")
    return t.data_ptr()


def n_alm(lmax: int) -> int:
    """Number of a_lm (m-major, m <= l <= lmax) of a real field."""
    return (lmax + 1) * (lmax + 2) // 2


def sht_alm2map(nside: int, lmax: int, d_alm, d_map, stream=None):
    """Synthesis on the GPU (ksc_sht_alm2map): d_alm complex128 device tensor of n_alm(lmax)
    entries (m-major), d_map float32 device tensor of 12 nside^2 pixels."""
    _check(_lib.ksc_sht_alm2map(int(nside), int(lmax), _dptr_alm(d_alm, lmax), _dptr(d_map),
                                _stream(stream)), "ksc_sht_alm2map")
    return d_map


def sht_map2alm(nside: int, lmax: int, d_map, d_alm, stream=None):
    """Analysis on the GPU (ksc_sht_map2alm), a_lm = (4 pi / Npix) sum_p m_p Y*_lm(p)."""
    _check(_lib.ksc_sht_map2alm(int(nside), int(lmax), _dptr(d_map), _dptr_alm(d_alm, lmax),
                                _stream(stream)), "ksc_sht_map2alm")
    return d_alm


def conv_harmonic(s: Split, d_in, d_out, add: bool = False, stream=None):
    """The split's harmonic half on the GPU (ksc_conv_harmonic); add=True adds it to d_out."""
    _check(_lib.ksc_conv_harmonic(s.handle, _dptr(d_in), _dptr(d_out), 1 if add else 0,
                                  _stream(stream)), "ksc_conv_harmonic")
    return d_out


def cost_model(**fields) -> CostModel:
    """The library's default cost model (ksc_cost_model_default), fields overridden."""
    m = CostModel()
    _check(_lib.ksc_cost_model_default(ctypes.byref(m)), "ksc_cost_model_default")
    for k, v in fields.items():
        setattr(m, k, float(v))
    return m


def eq8_cost_model(cores: int = 1) -> CostModel:
    """The host half as Eq. 8 prints it (160 s l_cut^2 l_max / 4096^3 on one 2.8 GHz
    core), spread over `cores` cores."""
    return cost_model(host_ms0=0.0, host_ms_eq8=160e3 / cores)


def cost_pairs(nside: int, theta_cut: float) -> float:
    return float(_lib.ksc_cost_pairs(int(nside), float(theta_cut)))


def cost_eval(m: CostModel, nside: int, l_cut: int, lmax: int, theta_cut: float):
    """(t_gpu_ms, t_host_ms) of one split under model m."""
    g, h = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ksc_cost_eval(ctypes.byref(m), int(nside), int(l_cut), int(lmax),
                              float(theta_cut), ctypes.byref(g), ctypes.byref(h)),
           "ksc_cost_eval")
    return g.value, h.value


def host_cost_ms(m: CostModel, l_cut, lmax) -> np.ndarray:
    """t_host (ms) for arrays of l_cut and l_max under model m."""
    lc, lm = np.broadcast_arrays(np.asarray(l_cut), np.asarray(lmax))
    return np.array([cost_eval(m, 1, int(a), int(b), 1e-3)[1] for a, b in zip(lc.ravel(),
                                                                             lm.ravel())])


def cost_fit_gpu(m: CostModel, nside, theta_cut, t_ms) -> CostModel:
    ns = np.ascontiguousarray(nside, dtype=np.int32)
    th = np.ascontiguousarray(theta_cut, dtype=np.float64)
    t = np.ascontiguousarray(t_ms, dtype=np.float64)
    _check(_lib.ksc_cost_fit_gpu(ns.ctypes.data, th.ctypes.data, t.ctypes.data, ns.size,
                                 ctypes.byref(m)), "ksc_cost_fit_gpu")
    return m


def cost_fit_host(m: CostModel, l_cut, lmax, t_ms) -> CostModel:
    lc = np.ascontiguousarray(l_cut, dtype=np.int32)
    lm = np.ascontiguousarray(lmax, dtype=np.int32)
    t = np.ascontiguousarray(t_ms, dtype=np.float64)
    _check(_lib.ksc_cost_fit_host(lc.ctypes.data, lm.ctypes.data, t.ctypes.data, lc.size,
                                  ctypes.byref(m)), "ksc_cost_fit_host")
    return m


def split_features(nside, fwhm_rad, l_cut, theta_cut_rad) -> np.ndarray:
    """Surrogate inputs (ksc_split_features), float32 (n, 4)."""
    ns, fw, lc, tc = np.broadcast_arrays(*(np.atleast_1d(np.asarray(v)) for v in
                                           (nside, fwhm_rad, l_cut, theta_cut_rad)))
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    fw = np.ascontiguousarray(fw, dtype=np.float64)
    lc = np.ascontiguousarray(lc, dtype=np.int32)
    tc = np.ascontiguousarray(tc, dtype=np.float64)
    out = np.empty((ns.size, 4), dtype=np.float32)
    _check(_lib.ksc_split_features(ns.size, ns.ctypes.data, fw.ctypes.data, lc.ctypes.data,
                                   tc.ctypes.data, out.ctypes.data), "ksc_split_features")
    return out


def scan_split(b_l, nside: int, cl_in=None, theta_lo=None, theta_hi=None, theta_step=None,
               bound=None, l_cut_fixed=None, linear_steps=None, cost: CostModel = None, **opts):
    """Sec. 2 scan (ksc_scan_split).  Returns (best_row_index or None, rows as dicts)."""
    b = np.ascontiguousarray(b_l, dtype=np.float64)
    lmax = b.size - 1
    so = ScanOpts()
    _check(_lib.ksc_scan_default_opts(ctypes.byref(so)), "ksc_scan_default_opts")
    for k, v in (("theta_lo", theta_lo), ("theta_hi", theta_hi), ("theta_step", theta_step),
                 ("bound", bound), ("l_cut_fixed", l_cut_fixed), ("linear_steps", linear_steps)):
        if v is not None:
            setattr(so, k, v)
    n_max = max(1, int(np.floor((so.theta_hi - so.theta_lo) / so.theta_step + 1e-9)) + 1)
    rows = (ScanRow * n_max)()
    cl = None if cl_in is None else np.ascontiguousarray(cl_in, dtype=np.float64)
    n, best = ctypes.c_int(), ctypes.c_int()
    _check(_lib.ksc_scan_split(b.ctypes.data, lmax, int(nside),
                               None if cl is None else cl.ctypes.data, ctypes.byref(so),
                               None if cost is None else ctypes.byref(cost),
                               ctypes.byref(default_opts(**opts)), rows, n_max, ctypes.byref(n),
                               ctypes.byref(best)), "ksc_scan_split")
    out = [{f: getattr(rows[i], f) for f, _ in ScanRow._fields_} for i in range(n.value)]
    return (best.value if best.value >= 0 else None), out
