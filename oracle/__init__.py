"""FP64 CPU oracle for the compact-kernel spherical convolution of arXiv:1409.4441.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_1409_4441_gb300``) never imports it, and this package
never imports the product path: the two share no code.  The only shared module
is the seeded input generator ``paper_1409_4441_gb300.inputs``, which holds no
arithmetic of the method.

What it computes, each function citing the passage of the paper it follows:

* ``split_lsq``: the weighted least-squares kernel split of Sec. 2, Eq. 1-5,
  solved by SVD with singular values below 1e-6 dropped.
* ``sigma_rms`` / ``frac_error`` / ``rel_error_l``: Eq. 2, Eq. 6 and Eq. 10.
* ``t_gpu_eq7`` / ``t_cpu_eq8`` / ``scan_split``: the cost models Eq. 7-8 and
  the scanning strategy of Sec. 2 (linear scan in theta_cut, binary search in
  l_cut, cheapest pair).
* ``brute_conv``: the real-space convolution (Sec. 1-2, Fig. 1's GPU half) as
  an all-pairs FP64 sum over every input pixel.
* ``map2alm`` / ``alm2map`` / ``sht_conv`` / ``alm2cl``: the harmonic
  convolution (Fig. 1's CPU half) and the power-spectrum extraction of Sec. 3.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, scipy special functions, exact identities or brute force on tiny
inputs; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np
from numpy.polynomial.legendre import leggauss

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ksc_oracle.c")
_LIB = os.path.join(_HERE, "libkscoracle.so")
_lib = None

ARCMIN = np.pi / (180.0 * 60.0)


def build(force: bool = False) -> str:
    """Compile the C half of the oracle (gcc, OpenMP) next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        vp = ctypes.c_void_p
        lib.orc_ring_table.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.orc_pix2vec.argtypes = [i64, vp]
        lib.orc_legendre_sum.argtypes = [i32, vp, i64, vp, vp, vp]
        lib.orc_brute_conv.argtypes = [i64, vp, i64, vp, i32, i32, vp, i64, vp, vp,
                                       dbl, dbl, vp, vp]
        lib.orc_count_pairs.argtypes = [i64, i64, vp, dbl, vp]
        lib.orc_lambda_table.argtypes = [i32, i32, i64, vp, vp]
        lib.orc_alm_analysis.argtypes = [i32, i32, i64, vp, vp, vp, dbl, vp]
        lib.orc_alm_synthesis.argtypes = [i32, i32, i64, vp, vp, vp, vp]
        for f in (lib.orc_ring_table, lib.orc_pix2vec, lib.orc_legendre_sum,
                  lib.orc_brute_conv, lib.orc_count_pairs, lib.orc_lambda_table,
                  lib.orc_alm_analysis, lib.orc_alm_synthesis):
            f.restype = i32
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# --------------------------------------------------------------------------
# HEALPix geometry (Gorski et al. 2005; nside 2048 data set of Sec. 2)
# --------------------------------------------------------------------------
def npix(nside: int) -> int:
    return 12 * nside * nside


def ring_table(nside: int):
    """Per-ring (z, sin theta, length, first pixel, phi of first pixel), rings 1..4n-1."""
    nr = 4 * nside - 1
    z = np.empty(nr); s = np.empty(nr); ln = np.empty(nr, np.int64)
    st = np.empty(nr, np.int64); ph = np.empty(nr)
    _check(_L().orc_ring_table(nside, _p(z), _p(s), _p(ln), _p(st), _p(ph)), "ring_table")
    return z, s, ln, st, ph


def pix2vec(nside: int) -> np.ndarray:
    """Unit vectors of all pixel centres, RING order, shape (Npix, 3)."""
    out = np.empty((npix(nside), 3))
    _check(_L().orc_pix2vec(nside, _p(out)), "pix2vec")
    return out


# --------------------------------------------------------------------------
# Kernel model and Legendre transforms (Eq. 1, Eq. 9)
# --------------------------------------------------------------------------
def gaussian_beam(lmax: int, fwhm_rad: float) -> np.ndarray:
    """Legendre transform of a Gaussian beam, B_l = exp(-l(l+1) sigma^2/2),
    sigma = FWHM / sqrt(8 ln 2) (the beam of Eq. 9, Sec. 3)."""
    sig = fwhm_rad / np.sqrt(8.0 * np.log(2.0))
    ell = np.arange(lmax + 1)
    return np.exp(-ell * (ell + 1) * sig * sig / 2.0)


def legendre_matrix(lmax: int, x) -> np.ndarray:
    """P_l(x_i) for l = 0..lmax by the three-term recurrence; shape (len(x), lmax+1)."""
    x = np.asarray(x, dtype=np.float64)
    P = np.empty((x.size, lmax + 1))
    P[:, 0] = 1.0
    if lmax >= 1:
        P[:, 1] = x
    for ell in range(1, lmax):
        P[:, ell + 1] = ((2 * ell + 1) * x * P[:, ell] - ell * P[:, ell - 1]) / (ell + 1)
    return P


def legendre_sum(c, z, deriv: bool = False):
    """K(z) = sum_l (2l+1)/(4 pi) c_l P_l(z) (and dK/dz): the real-space kernel
    whose Legendre transform 2 pi int K P_l dz is c_l (operator P_{l theta}, Eq. 1)."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.float64)
    K = np.empty_like(z)
    dK = np.empty_like(z) if deriv else None
    _check(_L().orc_legendre_sum(len(c) - 1, _p(c), z.size, _p(z), _p(K), _p(dK)),
           "legendre_sum")
    return (K, dK) if deriv else K


# --------------------------------------------------------------------------
# The weighted least-squares split (Sec. 2, Eq. 1-5) and its error (Eq. 2, 6, 10)
# --------------------------------------------------------------------------
def real_space_basis(lmax: int, theta_cut: float, oversample: int = 2):
    """Real-space unknowns of Eq. 4 and the columns P_{l,j} of Eq. 5.

    The z_cut unknowns are the nodes z_j of an ``oversample*(lmax+1)``-point
    Gauss-Legendre rule that lie inside the cap z >= cos(theta_cut).  Basis
    function j is the band-limited (l <= lmax) projection of a node at z_j with
    weight w_j, f_j(z) = w_j sum_l (2l+1)/2 P_l(z_j) P_l(z), truncated at
    theta_cut.  Column j of the Legendre operator is the exact transform of the
    truncated function, A_{l j} = 2 pi int_{cos theta_cut}^1 f_j P_l dz,
    evaluated with an (lmax+1)-point Gauss rule on [cos theta_cut, 1] (exact
    for the degree-2 lmax integrand).
    """
    zc = np.cos(theta_cut)
    xg, wg = leggauss(oversample * (lmax + 1))
    sel = xg >= zc
    zj, wj = xg[sel], wg[sel]
    xq, wq = leggauss(lmax + 1)
    zq = zc + (xq + 1.0) * (1.0 - zc) / 2.0
    wq = wq * (1.0 - zc) / 2.0
    ell = np.arange(lmax + 1)
    Pq = legendre_matrix(lmax, zq)
    Pj = legendre_matrix(lmax, zj)
    F = Pq @ (((2 * ell + 1) / 2.0)[:, None] * Pj.T) * wj[None, :]
    A = 2.0 * np.pi * (Pq.T @ (wq[:, None] * F))
    return zj, wj, Pj, A


def continuity_map(zj, wj, Pj, theta_cut: float, order: int):
    """Elimination matrix T (x = T t) that makes the truncated real-space kernel
    K_r = sum_j x_j f_j vanish at theta_cut (order 1), with zero slope there too
    (order 2).  Reading of Sec. 2's truncation "to a limit theta_cut": the
    compact kernel reaches zero continuously at the cut (a jump there makes the
    pixel sum of Sec. 3 miss or double-count boundary pixels).  The unknowns at
    the `order` nodes nearest the cut are expressed through the others:
    C_E x_E + C_F x_F = 0, rows of C = f_j(z_cut) and f_j'(z_cut), each f_j
    evaluated as the Legendre sum of its coefficients 2 pi w_j P_l(z_j)."""
    nz = zj.size
    if order <= 0 or nz <= order:
        return np.eye(nz), np.arange(nz)
    zc = np.cos(theta_cut)
    g, h = np.empty(nz), np.empty(nz)
    for j in range(nz):
        v, d = legendre_sum(2.0 * np.pi * wj[j] * Pj[j], zc, deriv=True)
        g[j], h[j] = v[0], d[0]
    E = np.argsort(np.abs(zj - zc))[:order]
    F = np.setdiff1d(np.arange(nz), E)
    Cm = np.vstack([g, h])[:order]
    T = np.zeros((nz, F.size))
    T[F, np.arange(F.size)] = 1.0
    T[E, :] = -np.linalg.solve(Cm[:, E], Cm[:, F])
    return T, F


def split_lsq(K, lcut: int, theta_cut: float, cl_in=None, oversample: int = 2,
              rcond: float = 1e-6, continuity: int = 2):
    """Eq. 3: A^T W A x = A^T W K_l, solved by SVD (Sec. 2).

    x = [Khat_l (l <= l_cut); Khat_theta (z_cut values)] (Eq. 4); A = [delta | P]
    (Eq. 5) with lmax+1 rows (l = 0..lmax); W = diag((2l+1) C_l^in) (Eq. 5 with
    the input spectrum of Eq. 2).  As in Sec. 2, the SVD is taken of the normal
    matrix A^T W A of Eq. 3 (columns of W^{1/2} A scaled to unit norm, so the
    cut is scale-free) and singular values below rcond (1e-6) times the largest
    are dropped.  With continuity 1 (2) the real-space kernel is constrained to
    vanish (with zero slope) at theta_cut by eliminating the unknowns nearest
    the cut (continuity_map); 0 leaves it free.

    Returns a dict with k_harm (l <= l_cut), x (real-space unknowns), the
    Legendre coefficients c_real (l <= lmax) of the real-space part before
    truncation, and K_tilde = Khat_l + P Khat_theta (Eq. 1).
    """
    K = np.asarray(K, dtype=np.float64)
    lmax = K.size - 1
    ell = np.arange(lmax + 1)
    C = np.ones(lmax + 1) if cl_in is None else np.asarray(cl_in, dtype=np.float64)
    zj, wj, Pj, A = real_space_basis(lmax, theta_cut, oversample)
    T, _ = continuity_map(zj, wj, Pj, theta_cut, continuity)
    nh = lcut + 1
    M = np.zeros((lmax + 1, nh + T.shape[1]))
    M[np.arange(nh), np.arange(nh)] = 1.0
    M[:, nh:] = A @ T
    sw = np.sqrt((2 * ell + 1) * C)
    B = sw[:, None] * M
    b = sw * K
    cn = np.linalg.norm(B, axis=0)
    cn[cn == 0] = 1.0
    Bn = B / cn
    N = Bn.T @ Bn                      # A^T W A, unit diagonal
    rhs = Bn.T @ b                     # A^T W K
    U, s, Vt = np.linalg.svd(N)
    keep = s > rcond * s[0]
    y = (Vt[keep].T @ ((U[:, keep].T @ rhs) / s[keep])) / cn
    k_harm = y[:nh]
    x = T @ y[nh:]
    c_real = 2.0 * np.pi * (Pj.T @ (wj * x))
    K_tilde = M @ y
    return dict(k_harm=k_harm, x=x, z_nodes=zj, w_nodes=wj, A=A, c_real=c_real,
                K_tilde=K_tilde, n_kept=int(keep.sum()), n_sv=int(s.size))


def split_sharp(K, lcut: int):
    """Literal split without a fit: Khat_l = K_l for l <= l_cut and the real-space
    part is the Legendre sum of the remaining l > l_cut (used for the split
    identity before truncation)."""
    K = np.asarray(K, dtype=np.float64)
    k_harm = K[: lcut + 1].copy()
    c_real = K.copy()
    c_real[: lcut + 1] = 0.0
    return dict(k_harm=k_harm, c_real=c_real)


def sigma_rms(K, K_tilde, cl_in=None) -> float:
    """Eq. 2: sigma_rms^2 = (1/4pi) sum_l (K_l - K~_l)^2 C_l^in (2l+1)."""
    K = np.asarray(K, float); Kt = np.asarray(K_tilde, float)
    ell = np.arange(K.size)
    C = np.ones(K.size) if cl_in is None else np.asarray(cl_in, float)
    return float(np.sqrt(np.sum((K - Kt) ** 2 * C * (2 * ell + 1)) / (4 * np.pi)))


def frac_error(K, K_tilde, cl_in=None, alpha: float = 5.0) -> float:
    """Eq. 6: sigma^2 = alpha^2 sigma_rms^2 / ((1/4pi) sum_l (2l+1) K_l^2 C_l^in)
    (denominator weighted by C_l^in like Eq. 2; alpha = 5 per Sec. 3)."""
    K = np.asarray(K, float)
    ell = np.arange(K.size)
    C = np.ones(K.size) if cl_in is None else np.asarray(cl_in, float)
    den = np.sum((2 * ell + 1) * K ** 2 * C) / (4 * np.pi)
    return float(alpha * sigma_rms(K, K_tilde, cl_in) / np.sqrt(den))


def rel_error_l(K, K_tilde) -> np.ndarray:
    """Eq. 10: sigma_l = log10 |1 - K~_l / K_l|."""
    with np.errstate(divide="ignore"):
        return np.log10(np.abs(1.0 - np.asarray(K_tilde) / np.asarray(K)))


def t_gpu_eq7(theta_cut_arcmin):
    """Eq. 7: GPU real-space cost on the paper's GTX 480, seconds."""
    return 0.0232 * np.asarray(theta_cut_arcmin) + 2.428


def t_cpu_eq8(lcut, lmax):
    """Eq. 8: single-core libpsht cost of the harmonic part, seconds."""
    return 160.0 * np.asarray(lcut, float) ** 2 * lmax / 4096.0 ** 3


def scan_split(K, theta_grid_rad, bound: float = 1e-5, cl_in=None, alpha: float = 5.0,
               t_gpu=None, t_cpu=None, oversample: int = 2, rcond: float = 1e-6,
               continuity: int = 2):
    """Sec. 2 scanning strategy: linear scan over theta_cut; for each, a binary
    search for the smallest l_cut meeting the Eq. 6 bound; then the pair with the
    least wall time max(t_gpu, t_cpu) (the two halves run concurrently, Fig. 1).

    Returns (best, table) where table lists (theta_cut, l_cut or None, error, cost).
    """
    K = np.asarray(K, float)
    lmax = K.size - 1
    t_gpu = t_gpu or (lambda th: float(t_gpu_eq7(th / ARCMIN)))
    t_cpu = t_cpu or (lambda lc: float(t_cpu_eq8(lc, lmax)))

    def err(lc, th):
        sp = split_lsq(K, lc, th, cl_in, oversample, rcond, continuity)
        return frac_error(K, sp["K_tilde"], cl_in, alpha)

    table = []
    for th in theta_grid_rad:
        lo, hi = 0, lmax - 1
        if err(hi, th) > bound:
            table.append((th, None, None, None))
            continue
        while lo < hi:
            mid = (lo + hi) // 2
            if err(mid, th) <= bound:
                hi = mid
            else:
                lo = mid + 1
        e = err(lo, th)
        table.append((th, lo, e, max(t_gpu(th), t_cpu(lo))))
    ok = [r for r in table if r[1] is not None]
    best = min(ok, key=lambda r: r[3]) if ok else None
    return best, table


# --------------------------------------------------------------------------
# Tabulated kernel (kernel-parity mode) and the brute-force convolution
# --------------------------------------------------------------------------
def chord_cut(theta_cut: float) -> float:
    return 2.0 * np.sin(0.5 * theta_cut)


def hermite_nodes(c, theta_cut: float, n_int: int):
    """Node values K(d_k) and slopes dK/dd at d_k = k h, h = d_cut / n_int, of the
    real-space kernel as a function of the chord d (z = 1 - d^2/2): the data of
    the cubic Hermite interpolant in d used by the tabulated convolution."""
    dc = chord_cut(theta_cut)
    d = np.arange(n_int + 1) * (dc / n_int)
    K, dKdz = legendre_sum(c, 1.0 - 0.5 * d * d, deriv=True)
    return K, -d * dKdz


def hermite_eval(tabK, tabD, theta_cut: float, d):
    """Evaluate the cubic Hermite interpolant of ``hermite_nodes`` at chord d."""
    n_int = len(tabK) - 1
    h = chord_cut(theta_cut) / n_int
    u = np.asarray(d, float) / h
    k = np.clip(np.floor(u).astype(np.int64), 0, n_int - 1)
    t = u - k
    h00 = 2 * t ** 3 - 3 * t ** 2 + 1
    h10 = t ** 3 - 2 * t ** 2 + t
    h01 = -2 * t ** 3 + 3 * t ** 2
    h11 = t ** 3 - t ** 2
    return h00 * tabK[k] + h10 * h * tabD[k] + h01 * tabK[k + 1] + h11 * h * tabD[k + 1]


def brute_conv(nside: int, m, theta_cut: float, c=None, table=None, out_pix=None,
               amb_eps: float = 1e-6):
    """All-pairs real-space convolution (Sec. 1-2):
    out_i = (4 pi/Npix) sum_{j: theta_ij <= theta_cut} K(theta_ij) m_j.

    Exactly one of ``c`` (K = Legendre sum of c, exact) or ``table`` = (tabK, tabD)
    (K = cubic Hermite interpolant in the chord) gives the kernel.  Returns
    (out, ambig) where ambig bounds the contribution of pairs lying within
    amb_eps (relative, in chord^2) of the cut.
    """
    m = np.ascontiguousarray(m, dtype=np.float64)
    assert m.size == npix(nside)
    if out_pix is None:
        n_out, op = npix(nside), None
    else:
        op = np.ascontiguousarray(out_pix, dtype=np.int64)
        n_out = op.size
    out = np.empty(n_out); amb = np.empty(n_out)
    if c is not None:
        cc = np.ascontiguousarray(c, dtype=np.float64)
        rc = _L().orc_brute_conv(nside, _p(m), n_out, _p(op), 0, cc.size - 1, _p(cc), 0,
                                 None, None, theta_cut, amb_eps, _p(out), _p(amb))
    else:
        tK = np.ascontiguousarray(table[0], dtype=np.float64)
        tD = np.ascontiguousarray(table[1], dtype=np.float64)
        rc = _L().orc_brute_conv(nside, _p(m), n_out, _p(op), 1, 0, None, tK.size - 1,
                                 _p(tK), _p(tD), theta_cut, amb_eps, _p(out), _p(amb))
    _check(rc, "brute_conv")
    return out, amb


def count_pairs(nside: int, theta_cut: float, out_pix=None) -> np.ndarray:
    """Number of input pixels within theta_cut of each listed output pixel."""
    op = None if out_pix is None else np.ascontiguousarray(out_pix, dtype=np.int64)
    n_out = npix(nside) if op is None else op.size
    cnt = np.empty(n_out, np.int64)
    _check(_L().orc_count_pairs(nside, n_out, _p(op), theta_cut, _p(cnt)), "count_pairs")
    return cnt


# --------------------------------------------------------------------------
# Spherical-harmonic transforms (the harmonic half of Fig. 1, spectra of Sec. 3)
# --------------------------------------------------------------------------
def alm_index(lmax: int, ell, m):
    return m * (2 * lmax + 1 - m) // 2 + ell


def n_alm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (2 * lmax + 2 - mmax) // 2


def lambda_table(lmax: int, z, mmax: int | None = None) -> np.ndarray:
    """Orthonormal associated Legendre functions lambda_lm(z), shape (npts, n_alm)."""
    mmax = lmax if mmax is None else mmax
    z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.float64)
    out = np.empty((z.size, n_alm(lmax, mmax)))
    _check(_L().orc_lambda_table(lmax, mmax, z.size, _p(z), _p(out)), "lambda_table")
    return out


def map2alm(nside: int, m, lmax: int, mmax: int | None = None) -> np.ndarray:
    """a_lm = (4 pi / Npix) sum_p m_p Y*_lm(p) (equal-weight quadrature), m >= 0."""
    mmax = lmax if mmax is None else mmax
    m = np.asarray(m, dtype=np.float64)
    z, s, ln, st, ph = ring_table(nside)
    nr = z.size
    F = np.empty((nr, mmax + 1), dtype=np.complex128)
    mm = np.arange(mmax + 1)
    for r in range(nr):
        L = int(ln[r])
        spec = np.fft.fft(m[st[r]: st[r] + L])
        F[r] = spec[mm % L] * np.exp(-1j * mm * ph[r])
    alm = np.empty(n_alm(lmax, mmax), dtype=np.complex128)
    _check(_L().orc_alm_analysis(lmax, mmax, nr, _p(z), _p(s), _p(F),
                                 4.0 * np.pi / npix(nside), _p(alm)), "alm_analysis")
    return alm


def alm2map(nside: int, alm, lmax: int, mmax: int | None = None) -> np.ndarray:
    """m_p = sum_lm a_lm Y_lm(p) for a real field.  Without the Condon-Shortley
    phase Y_{l,-m} = conj(Y_lm), so a real field has a_{l,-m} = conj(a_lm) and
    m_p = sum_l [a_l0 lambda_l0 + 2 Re sum_{m>0} a_lm Y_lm(p)]."""
    mmax = lmax if mmax is None else mmax
    alm = np.ascontiguousarray(alm, dtype=np.complex128)
    z, s, ln, st, ph = ring_table(nside)
    nr = z.size
    G = np.empty((nr, mmax + 1), dtype=np.complex128)
    _check(_L().orc_alm_synthesis(lmax, mmax, nr, _p(z), _p(s), _p(alm), _p(G)),
           "alm_synthesis")
    out = np.empty(npix(nside))
    mm = np.arange(mmax + 1)
    wgt = np.where(mm == 0, 1.0, 2.0)
    for r in range(nr):
        L = int(ln[r])
        H = np.zeros(L, dtype=np.complex128)
        np.add.at(H, mm % L, wgt * G[r] * np.exp(1j * mm * ph[r]))
        out[st[r]: st[r] + L] = np.real(np.fft.ifft(H) * L)
    return out


def sht_conv(nside: int, m, k_l, mmax: int | None = None) -> np.ndarray:
    """Harmonic convolution: alm2map(k_l * map2alm(m)) (Sec. 1, Fig. 1 CPU half)."""
    k_l = np.asarray(k_l, float)
    lmax = k_l.size - 1
    mmax = lmax if mmax is None else mmax
    alm = map2alm(nside, m, lmax, mmax)
    ell = np.concatenate([np.arange(mm, lmax + 1) for mm in range(mmax + 1)])
    return alm2map(nside, alm * k_l[ell], lmax, mmax)


def alm2cl(alm, lmax: int, mmax: int | None = None) -> np.ndarray:
    """C_l = (|a_l0|^2 + 2 sum_{m>0} |a_lm|^2) / (2l+1)."""
    mmax = lmax if mmax is None else mmax
    cl = np.zeros(lmax + 1)
    for mm in range(mmax + 1):
        base = alm_index(lmax, 0, mm)
        seg = np.abs(alm[base + mm: base + lmax + 1]) ** 2
        cl[mm:] += seg if mm == 0 else 2.0 * seg
    return cl / (2 * np.arange(lmax + 1) + 1)


def eps_cl(cl_split, cl_full, lmin: int = 0) -> float:
    """Fractional rms C_l error: sqrt(sum (2l+1)(C^s - C^f)^2 / sum (2l+1)(C^f)^2)."""
    cs = np.asarray(cl_split)[lmin:]; cf = np.asarray(cl_full)[lmin:]
    ell = np.arange(lmin, lmin + cs.size)
    return float(np.sqrt(np.sum((2 * ell + 1) * (cs - cf) ** 2) /
                         np.sum((2 * ell + 1) * cf ** 2)))
