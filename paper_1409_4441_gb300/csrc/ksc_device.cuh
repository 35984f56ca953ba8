// Device arithmetic shared by the convolution kernels.
//
// Chord -> table position, carried in "double-float" (an FP32 pair hi + lo,
// about 44 significant bits) so that the kernel argument is as accurate as the
// FP32 table itself.  For a pair of pixels on rings (z, s) and (z', s') that are
// dphi apart, chord^2 = A + B sin^2(dphi/2), A = (z - z')^2 + (s - s')^2,
// B = 4 s s'.  Scaling both by (n_int / d_cut)^2 gives the table position
// directly: u = d n_int / d_cut = sqrt(A' + B' sin^2 x), interval floor(u),
// offset u - floor(u), and the cut d <= d_cut is u^2 <= n_int^2.
#pragma once

#include <cuda_runtime.h>

namespace ksc {

struct DF {  // hi + lo
    float h, l;
};

// Split an FP64 value into an FP32 pair.
__host__ __device__ inline DF df_from_double(double v) {
    DF r;
    r.h = (float)v;
    r.l = (float)(v - (double)r.h);
    return r;
}

// sin(x) for x = xh + xl, |x| <= pi/2 + small, as a normalised pair
// (|lo| <= ulp(hi), as chord_to_table assumes).  sin x = x - x^3/6 + x^5 q(x^2)
// with q the Taylor series to x^13: x (exact) and -x^3/6 are carried in
// double-float, the smaller x^5 q term and the xl cos(x) correction in FP32.
__device__ __forceinline__ DF sin_df(float xh, float xl) {
    const float x2h = xh * xh;
    const float x2l = fmaf(xh, xh, -x2h);               // x^2 = x2h + x2l exactly
    const float x3h = xh * x2h;
    const float x3l = fmaf(xh, x2h, -x3h) + xh * x2l;    // x^3
    const float c6h = -0.16666667163372040f;             // -1/6 = c6h + c6l
    const float c6l = 4.9670538793415e-09f;
    const float t1h = x3h * c6h;
    const float t1l = fmaf(x3h, c6h, -t1h) + fmaf(x3h, c6l, x3l * c6h);  // -x^3/6
    float q = fmaf(1.6059043836821613e-10f, x2h, -2.5052108385441720e-08f);  // 1/13!, -1/11!
    q = fmaf(q, x2h, 2.7557319223985893e-06f);           //  1/9!
    q = fmaf(q, x2h, -1.9841269841269841e-04f);          // -1/7!
    q = fmaf(q, x2h, 8.3333333333333333e-03f);           //  1/5!
    const float rest = (x3h * x2h) * q;                  // x^5 q(x^2)
    const float c = fmaf(x2h, fmaf(x2h, 4.1666666666666664e-02f, -0.5f), 1.0f);  // ~cos
    // two-sum of the high parts, then normalise
    const float sh = xh + t1h;
    const float bp = sh - xh;
    const float e = (xh - (sh - bp)) + (t1h - bp);
    const float sl = e + t1l + rest + xl * c;
    DF s;
    s.h = sh + sl;
    s.l = (sh - s.h) + sl;
    return s;
}

// Table position for chord^2 * (n_int/d_cut)^2 = A + B sin^2(x).
// Returns false when the pair lies beyond the cut; otherwise interval i in
// [0, n_int - 1] and offset f (about [0, 1]).
__device__ __forceinline__ bool chord_to_table(DF A, DF B, DF s, float nint2, int n_int,
                                               int *i_out, float *f_out) {
    // s^2
    const float s2h = s.h * s.h;
    const float s2l = fmaf(2.0f * s.h, s.l, fmaf(s.h, s.h, -s2h));
    // B s^2
    const float ph = B.h * s2h;
    const float pl = fmaf(B.h, s2h, -ph) + fmaf(B.h, s2l, B.l * s2h);
    // D = A + B s^2 (two-sum on the high parts)
    const float dh = A.h + ph;
    const float bp = dh - A.h;
    const float e = (A.h - (dh - bp)) + (ph - bp);
    const float dl = e + A.l + pl;
    if (dh > nint2) return false;
    // u = sqrt(D): approximate reciprocal square root, then one double-float
    // Newton correction u = uh + (D - uh^2) / (2 uh)
    const float r = rsqrtf(fmaxf(dh, 1e-30f));
    const float uh = dh * r;
    const float ul = (fmaf(-uh, uh, dh) + dl) * (0.5f * r);
    // floor(uh) by the 1.5 * 2^23 rounding trick (uh < 2^22)
    const float t = (uh - 0.5f) + 12582912.0f;
    float fi = t - 12582912.0f;
    int i = __float_as_int(t) - 0x4B400000;
    const float top = (float)(n_int - 1);
    if (fi > top) { fi = top; i = n_int - 1; }
    if (fi < 0.0f) { fi = 0.0f; i = 0; }
    *i_out = i;
    *f_out = (uh - fi) + ul;
    return true;
}

// sin(x) as a normalised pair for |x| < 0.25: the Taylor tail x^3 q(x^2) (to
// x^9) in FP32 is below 2e-9 of sin x on this range, and cos x ~ 1 is enough
// for the xl correction.
__device__ __forceinline__ DF sin_df_small(float xh, float xl) {
    const float x2 = xh * xh;
    float q = fmaf(2.7557319223985893e-06f, x2, -1.9841269841269841e-04f);  //  1/9!, -1/7!
    q = fmaf(q, x2, 8.3333333333333333e-03f);                                //  1/5!
    q = fmaf(q, x2, -1.6666666666666667e-01f);                               // -1/3!
    const float tail = fmaf(xh * x2, q, xl);
    DF s;
    s.h = xh + tail;
    s.l = (xh - s.h) + tail;
    return s;
}

// chord_to_table for a table padded with an entry at n_int (the cut itself,
// u <= n_int, then needs no index clamp; u >= 0 always).
__device__ __forceinline__ bool chord_to_table_padded(DF A, DF B, DF s, float nint2, int *i_out,
                                                      float *f_out) {
    const float s2h = s.h * s.h;
    const float s2l = fmaf(2.0f * s.h, s.l, fmaf(s.h, s.h, -s2h));
    const float ph = B.h * s2h;
    const float pl = fmaf(B.h, s2h, -ph) + fmaf(B.h, s2l, B.l * s2h);
    const float dh = A.h + ph;
    const float bp = dh - A.h;
    const float e = (A.h - (dh - bp)) + (ph - bp);
    const float dl = e + A.l + pl;
    if (dh > nint2) return false;
    const float r = rsqrtf(fmaxf(dh, 1e-30f));
    const float uh = dh * r;
    const float ul = (fmaf(-uh, uh, dh) + dl) * (0.5f * r);
    const float t = (uh - 0.5f) + 12582912.0f;
    *i_out = __float_as_int(t) - 0x4B400000;
    *f_out = (uh - (t - 12582912.0f)) + ul;
    return true;
}

// Branch-free chord_to_table_padded: always returns a valid table position
// (beyond the cut, D is clamped to the cut, u = n_int, the padded entry) and
// reports whether the pair lies within the cut.  Straight-line code lets the
// compiler interleave several independent evaluations.
__device__ __forceinline__ bool chord_to_table_sel(DF A, DF B, DF s, float nint2, int *i_out,
                                                   float *f_out) {
    const float s2h = s.h * s.h;
    const float s2l = fmaf(2.0f * s.h, s.l, fmaf(s.h, s.h, -s2h));
    const float ph = B.h * s2h;
    const float pl = fmaf(B.h, s2h, -ph) + fmaf(B.h, s2l, B.l * s2h);
    const float dh0 = A.h + ph;
    const float bp = dh0 - A.h;
    const float e = (A.h - (dh0 - bp)) + (ph - bp);
    const float dl0 = e + A.l + pl;
    const bool in = dh0 <= nint2;
    const float dh = in ? dh0 : nint2;
    const float dl = in ? dl0 : 0.0f;
    const float r = rsqrtf(fmaxf(dh, 1e-30f));
    const float uh = dh * r;
    const float ul = (fmaf(-uh, uh, dh) + dl) * (0.5f * r);
    const float t = (uh - 0.5f) + 12582912.0f;
    *i_out = __float_as_int(t) - 0x4B400000;
    *f_out = (uh - (t - 12582912.0f)) + ul;
    return in;
}

__device__ __forceinline__ float hermite(const float4 c, float f) {
    return fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
}

} // namespace ksc
