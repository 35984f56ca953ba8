// Ring-pair geometry and kernel weights of the symmetric (cap) gather, shared
// by the FFMA kernel (conv_sym.cu) and the tensor-core kernel for map stacks
// (conv_sym_mma.cu).
//
// For output ring r (L pixels, phase flag t) and input ring q (L' pixels,
// phase t'), pixel k of r and pixel k' of q are dphi apart with
// dphi / 2 = N pi / (2 L L'), N = (2k + t) L' - (2k' + t') L an exact
// integer; the chord in table-position units is u^2 = A + B sin^2(dphi / 2)
// with the ring-pair constants A, B of the split (double-float, ksc_device.cuh).
#pragma once

#include "ksc_device.cuh"
#include "ksc_internal.h"

namespace ksc {

struct SymRing {  // one (output ring, input ring) pair
    DF A, B, c;
    float hw;     // half window in input pixels; < 0: no pixel within the cut
    int len, start, start_m, phase, small;
    // table in |N| (XInfo): cells of 2^shift integers, |N| <= ncut within the cut
    int shift, ncut, ncell;  // ncell 0: no table
    float inv;    // 2^-shift
    float pcl;    // ncut 2^-shift: the largest in-cut table position
    // odd-step table of the lockstep gather (XOdd): cells of 2 len / om in |N|
    int om, ooff, onct, oncut;  // onct 0: no table
    DF ocm;       // c / om
    float ohc;    // x extent of one cell
};

__device__ __forceinline__ int sym_pmod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Constants of (output ring r, input ring q); the pair is skipped (hw < 0) when
// skip_belt_inputs is set and q is a belt ring (the belt kernel covered it).
__device__ __forceinline__ SymRing load_sym_ring(const ConvPlan &P, int r, int q, int2 rg,
                                                 bool skip_belt_inputs) {
    const DevRing Qr = P.d_rings[q];
    const PairInfo pi = P.d_pairs[P.d_pair_base[r] + (q - rg.x)];
    SymRing g;
    g.A = DF{pi.Ah, pi.Al};
    g.B = DF{pi.Bh, pi.Bl};
    g.c = DF{pi.ch, pi.cl};
    g.hw = (skip_belt_inputs && q >= P.belt_lo && q <= P.belt_hi) ? -1.0f : pi.hw;
    g.len = Qr.len;
    g.start = Qr.start;
    g.start_m = P.d_rings[P.nrings - 1 - q].start;
    g.phase = Qr.phase;
    // |dphi / 2| < 0.25 over the whole (partial) window: the cheap sine
    g.small = (2.0f * pi.hw + 3.0f < (float)Qr.len) &&
              ((pi.hw + 1.0f) * 3.14159265f / (float)Qr.len < 0.25f);
    const XInfo xi = P.d_xinfo[P.d_pair_base[r] + (q - rg.x)];
    g.shift = xi.shift;
    g.ncut = xi.ncut;
    g.ncell = g.hw < 0.0f ? 0 : xi.ncell;
    g.inv = __int_as_float((127 - xi.shift) << 23);  // 2^-shift
    g.pcl = (float)xi.ncut * g.inv;
    const XOdd xo = P.d_xodd[P.d_pair_base[r] + (q - rg.x)];
    g.om = xo.m;
    g.ooff = xo.off;
    g.onct = g.hw < 0.0f ? 0 : xo.nct;
    g.oncut = xo.ncut;
    g.ocm = DF{xo.cmh, xo.cml};
    g.ohc = xo.hc;
    return g;
}

// Window [klo, khi] of input positions for output class k (one pixel of margin
// around |dphi| <= dphi_max; the whole ring, once, when a partial window could
// reach the ring's length).  The choice depends on the ring pair only, so both
// ends are nondecreasing in k and a CTA's union of windows runs from its first
// class's klo to its last class's khi.
__device__ __forceinline__ void sym_window(int k, int t, int L, const SymRing &g, long long *num,
                                           int *klo, int *khi) {
    const int L2 = g.len;
    *num = (long long)(2 * k + t) * L2 - (long long)g.phase * L;
    const float kc = (float)*num / (float)(2 * L);
    int lo, hi;
    if (2.0f * g.hw + 3.0f >= (float)L2) {
        lo = (int)floorf(kc) - L2 / 2;
        hi = lo + L2 - 1;
    } else {
        lo = (int)floorf(kc - g.hw);
        hi = (int)ceilf(kc + g.hw);  // hi - lo + 1 <= 2 hw + 3 < L2
    }
    *klo = lo;
    *khi = hi;
}

// Kernel weight of input position kp for the class whose exact integer at
// position 0 is num (Nf = num - 2 kp L as a float, exact below 2^24); zero
// outside [a, b] and beyond the cut.  Branch-free, so several evaluations
// interleave.
template <bool SMALL>
__device__ __forceinline__ float sym_weight(const ConvPlan &P, const SymRing &g, float Nf, int kp,
                                            int a, int b) {
    const float xh = Nf * g.c.h;
    const float xl = fmaf(Nf, g.c.h, -xh) + Nf * g.c.l;
    const DF sn = SMALL ? sin_df_small(xh, xl) : sin_df(xh, xl);
    int ti;
    float f;
    const bool in = chord_to_table_sel(g.A, g.B, sn, P.nint2, &ti, &f);
    const float wv = hermite(__ldg(&P.d_tab[min(ti, P.n_int)]), f);
    return (in && kp >= a && kp <= b) ? wv : 0.0f;
}

// Table of one ring pair (XInfo): the weight at cell boundary j, |N| = j 2^shift,
// x = |N| c, and its slope per cell, from the same double-float chord and K_r
// table as sym_weight.  Boundaries past the cut extrapolate the K_r table's last
// cubic, so the cell that holds the cut interpolates a smooth function.
__device__ __forceinline__ void xtab_node(const ConvPlan &P, const SymRing &g, int j, float *w,
                                          float *d, int off = 0) {
    const float Nf = (float)((j << g.shift) - off);  // exact: below 2^24
    const float xh = Nf * g.c.h;
    const float xl = fmaf(Nf, g.c.h, -xh) + Nf * g.c.l;
    const DF s = sin_df(xh, xl);
    const float s2h = s.h * s.h;
    const float s2l = fmaf(2.0f * s.h, s.l, fmaf(s.h, s.h, -s2h));
    const float ph = g.B.h * s2h;
    const float pl = fmaf(g.B.h, s2h, -ph) + fmaf(g.B.h, s2l, g.B.l * s2h);
    const float dh = g.A.h + ph;
    const float bp = dh - g.A.h;
    const float e = (g.A.h - (dh - bp)) + (ph - bp);
    const float dl = e + g.A.l + pl;
    const float rr = rsqrtf(fmaxf(dh, 1e-30f));
    const float uh = dh * rr;
    const float ul = (fmaf(-uh, uh, dh) + dl) * (0.5f * rr);
    const int i = max(0, min((int)floorf(uh), P.n_int - 1));
    const float f = (uh - (float)i) + ul;
    const float4 cf = __ldg(&P.d_tab[i]);
    *w = hermite(cf, f);
    const float dk = fmaf(f, fmaf(f, 3.0f * cf.w, 2.0f * cf.z), cf.y);  // dK/du
    // (the slope needs no more than the fast cosine: absolute error ~5e-7)
    const float dudx = g.B.h * s.h * __cosf(xh) * rr;  // rr = 1 / u
    *d = dk * dudx * (g.c.h * (float)(1 << g.shift));  // per cell: dx = 2^shift c
}

// The ring pair's table in shared memory, built by the T threads of a CTA:
// cell j holds the cubic coefficients (in the cell offset) from the weights and
// slopes at boundaries j and j + 1.  Each thread fills a run of consecutive
// cells (every boundary but the run's first evaluated once; an odd run length
// keeps a warp's 16-byte stores on distinct banks).
template <int T>
__device__ __forceinline__ void xtab_build(const ConvPlan &P, const SymRing &g, float4 *xt) {
    const int per = ((g.ncell + T - 1) / T) | 1;
    const int j0 = threadIdx.x * per, j1 = min(j0 + per, g.ncell);
    if (j0 >= j1) return;
    float w0, d0;
    xtab_node(P, g, j0, &w0, &d0);
    for (int j = j0; j < j1; ++j) {
        float w1, d1;
        xtab_node(P, g, j + 1, &w1, &d1);
        const float dw = w1 - w0;
        xt[j] = make_float4(w0, d0, fmaf(3.0f, dw, -fmaf(2.0f, d0, d1)),
                            fmaf(-2.0f, dw, d0 + d1));
        w0 = w1;
        d0 = d1;
    }
}

// The same table with its cell boundaries moved down by `off` integers, so that
// the last cell ends exactly at the cut: off = (-(ncut + 1)) mod 2^shift, cells
// 0 .. nct - 1 cover |N| + off in [j 2^shift, (j + 1) 2^shift), nct = (ncut + 1 +
// off) 2^-shift, and cell nct is zero.  A lookup at min(|N| + off, nct 2^shift)
// is then K_r within the cut and exactly 0 beyond it, with no test.
template <int T>
__device__ __forceinline__ void xtab_build_cut(const ConvPlan &P, const SymRing &g, float4 *xt,
                                               int off, int nct) {
    const int per = ((nct + T - 1) / T) | 1;
    const int j0 = threadIdx.x * per, j1 = min(j0 + per, nct);
    if (threadIdx.x == 0) xt[nct] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (j0 >= j1) return;
    float w0, d0;
    xtab_node(P, g, j0, &w0, &d0, off);
    for (int j = j0; j < j1; ++j) {
        float w1, d1;
        xtab_node(P, g, j + 1, &w1, &d1, off);
        const float dw = w1 - w0;
        xt[j] = make_float4(w0, d0, fmaf(3.0f, dw, -fmaf(2.0f, d0, d1)),
                            fmaf(-2.0f, dw, d0 + d1));
        w0 = w1;
        d0 = d1;
    }
}

// Node j of a ring pair's odd-step table (XOdd): the weight at table position
// P = j, |N| = (2 len j - off) / om (negative below the first in-range node:
// the weight is even in N), and its slope per cell, from the same double-float
// chord and K_r table as xtab_node.
__device__ __forceinline__ void xodd_node(const ConvPlan &P, const SymRing &g, int j, float *w,
                                          float *d) {
    const int n = 2 * g.len * j - g.ooff;  // < 2^31 (host check)
    const float nh = (float)n;
    const float nl = (float)(n - (int)nh);  // exact remainder
    const float xh = nh * g.ocm.h;
    const float xl = fmaf(nh, g.ocm.h, -xh) + fmaf(nh, g.ocm.l, nl * g.ocm.h);
    const DF s = sin_df(xh, xl);
    const float s2h = s.h * s.h;
    const float s2l = fmaf(2.0f * s.h, s.l, fmaf(s.h, s.h, -s2h));
    const float ph = g.B.h * s2h;
    const float pl = fmaf(g.B.h, s2h, -ph) + fmaf(g.B.h, s2l, g.B.l * s2h);
    const float dh = g.A.h + ph;
    const float bp = dh - g.A.h;
    const float e = (g.A.h - (dh - bp)) + (ph - bp);
    const float dl = e + g.A.l + pl;
    const float rr = rsqrtf(fmaxf(dh, 1e-30f));
    const float uh = dh * rr;
    const float ul = (fmaf(-uh, uh, dh) + dl) * (0.5f * rr);
    const int i = max(0, min((int)floorf(uh), P.n_int - 1));
    const float f = (uh - (float)i) + ul;
    const float4 cf = __ldg(&P.d_tab[i]);
    *w = hermite(cf, f);
    const float dk = fmaf(f, fmaf(f, 3.0f * cf.w, 2.0f * cf.z), cf.y);  // dK/du
    const float dudx = g.B.h * s.h * __cosf(xh) * rr;
    *d = dk * dudx * g.ohc;
}

// The odd-step table in shared memory, built by the T threads of a CTA: cells
// 0 .. onct-1 from the weights and slopes at their two boundaries, cell onct zero.
template <int T>
__device__ __forceinline__ void xodd_build(const ConvPlan &P, const SymRing &g, float4 *xt) {
    const int nct = g.onct;
    const int per = ((nct + T - 1) / T) | 1;
    const int j0 = threadIdx.x * per, j1 = min(j0 + per, nct);
    if (threadIdx.x == 0) xt[nct] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (j0 >= j1) return;
    float w0, d0;
    xodd_node(P, g, j0, &w0, &d0);
    for (int j = j0; j < j1; ++j) {
        float w1, d1;
        xodd_node(P, g, j + 1, &w1, &d1);
        const float dw = w1 - w0;
        xt[j] = make_float4(w0, d0, fmaf(3.0f, dw, -fmaf(2.0f, d0, d1)),
                            fmaf(-2.0f, dw, d0 + d1));
        w0 = w1;
        d0 = d1;
    }
}

// Cubic of table position p = |N| 2^-shift (exact) from the table xt: cell
// floor(p), offset p - floor(p).  p < 2^22, so adding 1.5 * 2^23 rounded
// downward gives floor(p) in the low mantissa bits.
__device__ __forceinline__ float xtab_at(const float4 *xt, float p) {
    const float t = __fadd_rd(p, 12582912.0f);
    const float4 cf = xt[__float_as_uint(t) - 0x4B400000u];
    const float f = p - (t - 12582912.0f);
    return hermite(cf, f);
}

// Weight of the pixel pair with exact integer Nf from the table xt; zero beyond
// the cut (the position is clamped into the table first).
__device__ __forceinline__ float xtab_weight(const float4 *xt, const SymRing &g, float Nf) {
    const float an = fabsf(Nf);
    const float v = xtab_at(xt, fminf(an * g.inv, g.pcl));
    return an <= (float)g.ncut ? v : 0.0f;
}

} // namespace ksc
