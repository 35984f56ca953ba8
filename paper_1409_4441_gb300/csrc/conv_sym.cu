// Real-space convolution, symmetric gather for ring pairs outside the
// circulant belt path (polar caps, and belt rings whose disc reaches a cap).
//
// HEALPix RING geometry has a 16-element symmetry group that preserves every
// chord: quarter turns about the polar axis (pixel k of a ring of L = 4Q pixels
// maps to k + Q), the north/south mirror z -> -z (ring r maps to ring 4n-2-r
// with the same pixel phases) and the reflection phi -> pi/2 - phi (pixel k of
// a ring with phase flag t maps to Q - k - t).  So one kernel evaluation
// w(k, k') serves sixteen pixel pairs:
//
//   out[r,   k  + qQ] += w m[r',   k'  + qQ']      q = 0..3
//   out[r,   kb + qQ] += w m[r',   kb' + qQ']      kb = Q - k - t, kb' = Q' - k' - t'
//   and the same on the mirror rings r_s, r'_s.
//
// One thread owns C consecutive reflection classes {k, kb} of first-quarter
// positions of a northern ring (a class of one when kb coincides with k up to a
// quarter turn) and produces all their images (no mirror on the equator ring,
// which is its own mirror image).  Per input ring the CTA stages, for the union
// of its threads' windows, the sixteen image sequences m[image(k')] in shared
// memory so that every image of input position k' sits at the same offset.
//
// A weight depends on the pixel pair only through the exact integer
// N = (2k + t) L' - (2k' + t') L (dphi / 2 = N pi / (2 L L')).  Per input ring
// the CTA builds the ring pair's odd-step weight table (XOdd: cubic cells of
// 2 L' / m in |N|, m odd, ksc_sym.cuh) in shared memory, and the eight lanes of
// each quarter warp walk the same input positions (the lockstep path below):
// their table positions then differ by whole cells, m C per lane (an odd
// number), so a quarter's eight 16-byte cell loads fall in eight different bank
// groups, and one exact rational position per quarter serves all its weights.
// A weight is a cell load and three FMAs, exactly zero beyond the cut with no
// test; four positions of a thread then take one 16-byte shared load per image
// feeding 4 C FFMAs.  Ring pairs without a table (whole-ring windows, or more
// cells than a CTA holds) evaluate the double-float chord and the K_r table per
// pair (ksc_device.cuh).  FP32 partial sums are Kahan-folded into the totals
// every 64 positions, and every 8 around the kernel's centre.
#include <cstdint>

#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_sym.cuh"

namespace ksc {
namespace {

constexpr int kRingChunk = 32;  // ring-pair constants staged per pass
constexpr int kImg = 16;        // 4 rotations x {north, south} x {direct, reflected}
constexpr int kPair = 8;        // image pairs (north, south mirror): FP32x2 operands
// FP32 partial sums fold into the compensated sums every kFold quads (64
// positions), and every kFoldNear quads around the kernel's centre, where the
// largest terms are: a term's partial then takes few roundings at its size.
constexpr int kFold = 16;
constexpr int kFoldNear = 2;
constexpr int kFoldPair = 4;    // per-pair path: every 16 positions
// Tile shape: T threads of C classes each, SPAN staged input positions per
// segment (each image row padded by 4 floats), MINB resident CTAs per SM the
// register budget is set for, XCAP table cells in dynamic shared memory.
template <int T_, int C_, int SPAN_, int MINB_, int XCAP_> struct SymShape {
    static constexpr int T = T_, C = C_, kSpan = SPAN_, MINB = MINB_, kXCap = XCAP_;
    static constexpr int kStride = SPAN_ + 4;
    static constexpr int kClasses = T_ * C_;
    static constexpr size_t kDynSmem = sizeof(float4) * (size_t)XCAP_;
};
using ShapeC3 = SymShape<128, 3, 640, 2, kXCap>;    // variant 0: 384 classes per item
using ShapeSmall = SymShape<128, 1, 448, 3, 2048>;  // variant 1: 128 classes, 3 CTAs per SM
using ShapeWide = SymShape<128, 1, 448, 2, kXCap>;  // variant 2: 128 classes, full tables
static_assert(ShapeC3::kSpan % 4 == 0 && ShapeSmall::kSpan % 4 == 0, "quad-aligned spans");

// Kahan step on a pair of sums, with the compensation carried in the partial:
// the partial starts from the low part the previous step lost (rather than
// from zero), so one step is t = s + p, p = p - (t - s), s = t, every operation
// rounded to nearest (t - s = fma(s, -1, t)).
__device__ __forceinline__ void kahan2(float2 &sum, float2 &part) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 t = __fadd2_rn(sum, part);
    part = __ffma2_rn(__ffma2_rn(sum, m1, t), m1, part);
    sum = t;
}

// floor(a / b), ceil(a / b) for b > 0
__device__ __forceinline__ int floor_div(int a, int b) {
    const int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int ceil_div(int a, int b) {
    const int q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}

// The sixteen images of one quad of positions for the C classes of a thread.  The
// staged images are stored as eight (north, south mirror) pairs interleaved by
// position, so one 16-byte shared load gives two positions of a pair, and each
// multiply-add is a paired FP32 FMA (two images, one weight): 32 paired FMAs per
// class and quad.  (On the equator ring, its own mirror, the south halves hold
// zeros and their sums are never written.)
template <class S>
__device__ __forceinline__ void fma_quad(const float *st, int j, const float4 *w, float2 *part) {
#pragma unroll
    for (int r = 0; r < kPair; ++r) {
        const float *row = st + r * 2 * S::kStride + 2 * j;
        const float4 a = *reinterpret_cast<const float4 *>(row);
        const float4 b = *reinterpret_cast<const float4 *>(row + 4);
#pragma unroll
        for (int c = 0; c < S::C; ++c) {
            float2 p = part[c * kPair + r];
            p = __ffma2_rn(make_float2(w[c].x, w[c].x), make_float2(a.x, a.y), p);
            p = __ffma2_rn(make_float2(w[c].y, w[c].y), make_float2(a.z, a.w), p);
            p = __ffma2_rn(make_float2(w[c].z, w[c].z), make_float2(b.x, b.y), p);
            p = __ffma2_rn(make_float2(w[c].w, w[c].w), make_float2(b.z, b.w), p);
            part[c * kPair + r] = p;
        }
    }
}

template <class S>
__device__ __forceinline__ void fold(float2 *sum, float2 *part) {
#pragma unroll
    for (int i = 0; i < S::C * kPair; ++i) kahan2(sum[i], part[i]);
}

// Stage the sixteen image sequences of input positions s0 .. s0 + span - 1 as
// eight (north, south) pairs: pair r < 4 holds quarter turn r of the direct
// images, pair 4 + r of the reflected ones; element (r, j) at st[2 (r kStride + j)].
template <class S, bool MIRROR>
__device__ __forceinline__ void stage(const SymRing &g, const float *__restrict__ m, float *st,
                                      int s0, int span) {
    constexpr int kStride = S::kStride;
    const int L2 = g.len, Q2 = L2 / 4;
    for (int j = threadIdx.x; j < span; j += S::T) {
        const int kp = s0 + j;
        const int idx = sym_pmod(kp, L2);
        const int idr = sym_pmod(Q2 - kp - g.phase, L2);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            int ia = idx + qq * Q2;
            if (ia >= L2) ia -= L2;
            int ib = idr + qq * Q2;
            if (ib >= L2) ib -= L2;
            const float an = __ldg(m + g.start + ia), bn = __ldg(m + g.start + ib);
            const float as = MIRROR ? __ldg(m + g.start_m + ia) : 0.0f;
            const float bs = MIRROR ? __ldg(m + g.start_m + ib) : 0.0f;
            *reinterpret_cast<float2 *>(st + 2 * (qq * kStride + j)) = make_float2(an, as);
            *reinterpret_cast<float2 *>(st + 2 * ((4 + qq) * kStride + j)) = make_float2(bn, bs);
        }
    }
}

// ---------------------------------------------------------------------------
// Lockstep table path.  The eight lanes of a quarter warp own classes
// kQ + C l .. kQ + C l + C - 1 (l = 0..7) and walk the same input positions, a
// quad of four at a time, from the first in-cut position of the quarter's first
// class to the last of its last class; the four quarters of a warp walk in step
// (each from its own start), so every lane reads the same image float4 as the
// other lanes of its quarter.  At position p the quarter's first class has
// N = NQ(p) = numQ - 2 L p, and class c of lane l has N = NQ + 2 L' (C l + c).
// The ring pair's odd-step table (XOdd) has cells of 2 L' / m in |N|, so with
// P = (|N| m + off) / (2 L'):
//   N >= 0:  P = PQ + m (C l + c),   PQ = (NQ m + off) / (2 L'),
//   N <= 0:  P = PN - m (C l + c),   PN = (-NQ m + off) / (2 L'),
// one rational position per quarter and position, shared by its 8 C weights:
// the offset in the cell is common, the cells of the eight lanes are m C apart
// (odd), and the quarter's eight 16-byte cell loads fall in eight different bank
// groups.  PQ and PN are carried exactly as integer + remainder / (2 L') (the
// remainder an integer-valued float below 2^16).  Quads where every lane has
// N >= 0 (or <= 0) take one state; the few quads where the quarter's lanes
// straddle N = 0 take both and choose per weight.  Positions beyond a class's cut
// read the zero cell (indices clamped to it), so no weight needs a mask.
// ---------------------------------------------------------------------------

// Exact position state integer + remainder / D (0 <= remainder < D).
struct OddPos {
    int a;    // floor of the position
    float R;  // remainder (an integer, as a float)
};

__device__ __forceinline__ OddPos odd_pos(int M, int D) {
    const int a = floor_div(M, D);
    return OddPos{a, (float)(M - a * D)};
}

// Step constants: one position (N down by 2 L) moves PQ down and PN up by
// (2 L m) / D = q1 + r1 / D.
struct OddStep {
    int q1, q2, D2;    // D2 = 2 L' (N between consecutive classes)
    unsigned nct;  // the zero cell
    float r1, r2, Df, invD;
};

__device__ __forceinline__ void pos_down(OddPos &s, const OddStep &k) {
    s.R -= k.r1;
    const bool b = s.R < 0.0f;
    s.R = b ? s.R + k.Df : s.R;
    s.a -= k.q1 + (b ? 1 : 0);
}
__device__ __forceinline__ void pos_up(OddPos &s, const OddStep &k) {
    s.R += k.r1;
    const bool b = s.R >= k.Df;
    s.R = b ? s.R - k.Df : s.R;
    s.a += k.q1 + (b ? 1 : 0);
}
__device__ __forceinline__ void pos_down2(OddPos &s, const OddStep &k) {
    s.R -= k.r2;
    const bool b = s.R < 0.0f;
    s.R = b ? s.R + k.Df : s.R;
    s.a -= k.q2 + (b ? 1 : 0);
}
__device__ __forceinline__ void pos_up2(OddPos &s, const OddStep &k) {
    s.R += k.r2;
    const bool b = s.R >= k.Df;
    s.R = b ? s.R - k.Df : s.R;
    s.a += k.q2 + (b ? 1 : 0);
}

__device__ __forceinline__ float odd_weight(const float4 *xt, int idx, unsigned nct, float f) {
    return hermite(xt[min((unsigned)idx, nct)], f);
}

// Weights of one quad, every lane's N of one sign: SIGN > 0 walks PQ (kk[c] =
// m (C l + c) added), SIGN < 0 walks PN (subtracted).  The state advances by the
// quad's four positions.
template <int C, int SIGN>
__device__ __forceinline__ void quad_fast(const float4 *xt, OddPos &s, const OddStep &k,
                                          const int *kk, float4 *w) {
    // positions 0..3 from the quad start with a dependence depth of two steps
    OddPos p[4];
    p[0] = s;
    p[1] = s;
    p[2] = s;
    if (SIGN > 0) { pos_down(p[1], k); pos_down2(p[2], k); }
    else { pos_up(p[1], k); pos_up2(p[2], k); }
    p[3] = p[2];
    s = p[2];
    if (SIGN > 0) { pos_down(p[3], k); pos_down2(s, k); }
    else { pos_up(p[3], k); pos_up2(s, k); }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const float f = p[d].R * k.invD;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float v = odd_weight(xt, SIGN > 0 ? p[d].a + kk[c] : p[d].a - kk[c], k.nct, f);
            if (d == 0) w[c].x = v;
            else if (d == 1) w[c].y = v;
            else if (d == 2) w[c].z = v;
            else w[c].w = v;
        }
    }
}

// Weights of one quad whose lanes straddle N = 0: per weight the sign of the
// lane's N = NQ + 2 L' (C l + c) (N >= 0 while NQ >= thr0 - c 2 L').
template <int C>
__device__ __forceinline__ void quad_mixed(const float4 *xt, OddPos &sp, OddPos &sn, int &NQ,
                                           int Dl, const OddStep &k, const int *kk,
                                           int thr0, float4 *w) {
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const float fp = sp.R * k.invD, fn = sn.R * k.invD;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const bool pos = NQ >= thr0 - c * k.D2;
            const float v = odd_weight(xt, pos ? sp.a + kk[c] : sn.a - kk[c], k.nct,
                                       pos ? fp : fn);
            if (d == 0) w[c].x = v;
            else if (d == 1) w[c].y = v;
            else if (d == 2) w[c].z = v;
            else w[c].w = v;
        }
        pos_down(sp, k);
        pos_up(sn, k);
        NQ -= Dl;
    }
}

// Quads j in [ja, jb) of one regime for this lane's quarter (first position
// p0 = QA4 + 4 ja, local offset in the staged segment p0 - s0).
template <class S, bool MIRROR, int SIGN>
__device__ __forceinline__ void run_fast(const float4 *xt, const float *st, int loc, int nquads,
                                         OddPos s, const OddStep &k, const int *kk, float2 *sum,
                                         float2 *part, int &nfold) {
    constexpr int C = S::C;
    for (int q = 0; q < nquads; ++q) {
        float4 w[C];
        quad_fast<C, SIGN>(xt, s, k, kk, w);
        fma_quad<S>(st, loc, w, part);
        loc += 4;
        if (++nfold == kFold) {
            nfold = 0;
            fold<S>(sum, part);
        }
    }
}

template <class S, bool MIRROR>
__device__ __forceinline__ void run_mixed(const float4 *xt, const float *st, int loc, int nquads,
                                          OddPos sp, OddPos sn, int NQ, int Dl, const OddStep &k,
                                          const int *kk, int thr0, float2 *sum,
                                          float2 *part, int &nfold) {
    constexpr int C = S::C;
    // the quads where some lane's N changes sign hold every lane's centre: the
    // partial before them ends here, theirs fold every kFoldNear quads, and the
    // next kFoldNear quads (the last lanes' terms just past the centre) end theirs
    fold<S>(sum, part);
    for (int q = 0; q < nquads; ++q) {
        float4 w[C];
        quad_mixed<C>(xt, sp, sn, NQ, Dl, k, kk, thr0, w);
        fma_quad<S>(st, loc, w, part);
        loc += 4;
        if ((q + 1) % kFoldNear == 0) fold<S>(sum, part);
    }
    if (nquads % kFoldNear != 0) fold<S>(sum, part);
    nfold = kFold - kFoldNear;
}

// One ring pair through the lockstep path.  Returns false (before any work, and
// the same in every thread) when a warp's quarters spread wider than a staged
// segment; the caller then takes the per-pair path.
template <class S, bool MIRROR>
__device__ __forceinline__ bool lockstep_pair(const ConvPlan &P, const SymRing &g, int c0,
                                              int n_cls, int t, int L,
                                              const float *__restrict__ m, float *st,
                                              float4 *xt, int *sW, float2 *sum,
                                              float2 *part) {
    constexpr int T = S::T, C = S::C, kSpan = S::kSpan, NW = T / 32;
    const int tid = threadIdx.x, wid = tid >> 5, ql = tid & 7;
    const int L2 = g.len;
    const int D = 2 * L2, Dl = 2 * L;
    const int ncut = g.oncut;
    // this lane's quarter: classes kQ .. kQ + 8 C - 1 (those below n_cls exist); class
    // integers fit in int32 (checked by the caller)
    const int kQ = c0 + C * (tid & ~7);
    const int kQe = min(kQ + 8 * C - 1, n_cls - 1);
    const int numQ = (2 * kQ + t) * L2 - g.phase * L;
    const int numQe = numQ + 2 * L2 * (kQe - kQ);
    // in-cut positions of the quarter's existing classes: |num - 2 L p| <= ncut
    const int QA = ceil_div(numQ - ncut, Dl), QB = floor_div(numQe + ncut, Dl);
    const int QA4 = QA & ~3;
    const int Jq = (kQ < n_cls && QB >= QA) ? ((QB - QA4) >> 2) + 1 : 0;
    const int Jw = __reduce_max_sync(0xffffffffu, Jq);
    const int loW = __reduce_min_sync(0xffffffffu, Jq > 0 ? QA4 : 0x7fffffff);
    const int hiW = __reduce_max_sync(0xffffffffu, Jq > 0 ? QA4 : (int)0x80000000);
    // N of the quarter's first class at its first position (small: near the cut;
    // the products wrap, the difference is exact)
    const int NQ0 = (int)((unsigned)numQ - (unsigned)Dl * (unsigned)QA4);
    // regimes over quads j (p = QA4 + 4 j): every lane's N >= 0 while NQ(p + 3) >= 0;
    // every lane's N <= 0 once NQ(p) + 2 L' (8 C - 1) <= 0
    int jPq = Jw, jNq = 0;
    if (Jq > 0) {
        jPq = max(0, min(Jw, floor_div(NQ0 - 3 * Dl, 4 * Dl) + 1));
        jNq = max(0, min(Jw, ceil_div(NQ0 + 2 * L2 * (8 * C - 1), 4 * Dl)));
    }
    const int jP = __reduce_min_sync(0xffffffffu, jPq);
    const int jN = max(jP, __reduce_max_sync(0xffffffffu, jNq));

    __syncthreads();  // the previous ring pair's table, segment and sW reads are done
    if ((tid & 31) == 0) {
        sW[4 * wid + 0] = Jw;
        sW[4 * wid + 1] = loW;
        sW[4 * wid + 2] = hiW;
    }
    xodd_build<T>(P, g, xt);
    __syncthreads();
    int lo = 0x7fffffff, hi = (int)0x80000000;
    bool wide = false;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int J = sW[4 * w], l = sW[4 * w + 1], h = sW[4 * w + 2];
        if (J > 0) {
            lo = min(lo, l);
            hi = max(hi, h + 4 * J - 1);
            wide = wide || (h - l + 8 > kSpan);
        }
    }
    if (wide) return false;
    if (lo > hi) return true;  // no class of this item has a pair within the cut

    // per lane: table offsets of its classes, step constants
    int kk[C];
#pragma unroll
    for (int c = 0; c < C; ++c) kk[c] = g.om * (C * ql + c);
    const int thr0 = -2 * L2 * C * ql;  // lane's N >= 0 while NQ >= thr0 - c 2 L'
    OddStep k;
    {
        const int st1 = Dl * g.om;
        k.q1 = st1 / D;
        k.r1 = (float)(st1 - k.q1 * D);
        k.q2 = (2 * st1) / D;
        k.r2 = (float)(2 * st1 - k.q2 * D);
        k.Df = (float)D;
        k.D2 = D;
        k.invD = 1.0f / (float)D;
        k.nct = (unsigned)g.onct;
    }
    int jnext = 0;  // the warp's next quad
    int nfold = 0;
    const bool single = hi - lo + 1 <= kSpan;  // one segment: no reduction between segments
    for (int s0 = lo;;) {
        const int span = min(kSpan, ((hi - s0 + 1) + 3) & ~3);
        stage<S, MIRROR>(g, m, st, s0, span);
        __syncthreads();
        // quads of this warp inside the segment: every quarter's quad within it
        int jB = jnext;
        if (Jw > 0 && jnext < Jw)
            jB = max(jnext, min(Jw, floor_div(s0 + span - 4 - hiW, 4) + 1));
        if (Jq > 0 && jB > jnext) {
            const int loc0 = QA4 + 4 * jnext - s0;
            // [jnext, jB) split into N >= 0, mixed and N <= 0 quads
            const int e1 = min(jB, max(jnext, jP));
            const int e2 = min(jB, max(e1, jN));
            if (e1 > jnext) {
                const int NQ = NQ0 - 4 * Dl * jnext;
                run_fast<S, MIRROR, 1>(xt, st, loc0, e1 - jnext, odd_pos(NQ * g.om + g.ooff, D),
                                       k, kk, sum, part, nfold);
            }
            if (e2 > e1) {
                const int NQ = NQ0 - 4 * Dl * e1;
                run_mixed<S, MIRROR>(xt, st, loc0 + 4 * (e1 - jnext), e2 - e1,
                                     odd_pos(NQ * g.om + g.ooff, D),
                                     odd_pos(-NQ * g.om + g.ooff, D), NQ, Dl, k, kk, thr0, sum,
                                     part, nfold);
            }
            if (jB > e2) {
                const int NQ = NQ0 - 4 * Dl * e2;
                run_fast<S, MIRROR, -1>(xt, st, loc0 + 4 * (e2 - jnext), jB - e2,
                                        odd_pos(-NQ * g.om + g.ooff, D), k, kk, sum, part,
                                        nfold);
            }
        }
        if (single) break;
        jnext = jB;
        // the next segment starts at the first quad some warp has left
        if ((tid & 31) == 0) sW[4 * wid + 3] = jnext < Jw ? loW + 4 * jnext : 0x7fffffff;
        __syncthreads();
        int nxt = 0x7fffffff;
#pragma unroll
        for (int w = 0; w < NW; ++w) nxt = min(nxt, sW[4 * w + 3]);
        if (nxt == 0x7fffffff) break;
        __syncthreads();  // every thread has read sW and consumed the segment
        s0 = nxt;
    }
    fold<S>(sum, part);
    return true;
}

// Per-pair path (no table): the four kernel weights of quad kq (zero outside
// [a, b] and beyond the cut); MODE 0: double-float chord with the general sine,
// 1: with the small-angle sine.  Straight-line code: the evaluations interleave.
template <int MODE>
__device__ __forceinline__ float4 quad_weights(const ConvPlan &P, const SymRing &g, int kq,
                                               int a, int b, long long num, int L) {
    const float N0 = (float)(num - 2LL * kq * L);  // exact integer below 2^24
    const float step = (float)(2 * L);
    return make_float4(sym_weight<MODE == 1>(P, g, N0, kq, a, b),
                       sym_weight<MODE == 1>(P, g, N0 - step, kq + 1, a, b),
                       sym_weight<MODE == 1>(P, g, N0 - 2.0f * step, kq + 2, a, b),
                       sym_weight<MODE == 1>(P, g, N0 - 3.0f * step, kq + 3, a, b));
}

// Positions a..b of one segment for classes c = 0..C-1 with windows
// [lo[c], hi[c]] (num of class c = num0 + 2 c L2).
template <class S, int MODE>
__device__ __forceinline__ void acc_pairs(const ConvPlan &P, const SymRing &g, const float *st,
                                          int s0, int a, int b, long long num0, int L,
                                          const int *lo, const int *hi, float2 *sum,
                                          float2 *part) {
    constexpr int C = S::C;
    int nq = 0;
    for (int kq = s0 + ((a - s0) & ~3); kq <= b; kq += 4) {
        // (rare: one class at a time, each loading the images again)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float4 w[C];
            w[0] = quad_weights<MODE>(P, g, kq, lo[c], hi[c], num0 + 2LL * c * g.len, L);
#pragma unroll
            for (int r = 0; r < kPair; ++r) {
                const float *row = st + r * 2 * S::kStride + 2 * (kq - s0);
                const float4 va = *reinterpret_cast<const float4 *>(row);
                const float4 vb = *reinterpret_cast<const float4 *>(row + 4);
                float2 p = part[c * kPair + r];
                p = __ffma2_rn(make_float2(w[0].x, w[0].x), make_float2(va.x, va.y), p);
                p = __ffma2_rn(make_float2(w[0].y, w[0].y), make_float2(va.z, va.w), p);
                p = __ffma2_rn(make_float2(w[0].z, w[0].z), make_float2(vb.x, vb.y), p);
                p = __ffma2_rn(make_float2(w[0].w, w[0].w), make_float2(vb.z, vb.w), p);
                part[c * kPair + r] = p;
            }
        }
        if (++nq == kFoldPair) {
            nq = 0;
            fold<S>(sum, part);
        }
    }
    fold<S>(sum, part);
}

template <class S, bool MIRROR>
__device__ __forceinline__ void sym_item(const ConvPlan &P, int r, int c0, int n_cls,
                                         bool skip_belt_inputs, bool add, int band_lo,
                                         int band_hi, const float *__restrict__ m,
                                         float *__restrict__ o, SymRing *sR, float *st,
                                         float4 *xt, int *sW, int *__restrict__ err) {
    constexpr int C = S::C, kSpan = S::kSpan;
    const int tid = threadIdx.x;
    const DevRing R = P.d_rings[r];
    const int L = R.len, Q = L / 4, t = R.phase;
    const int2 rg = P.d_range[r];
    const int k0 = c0 + C * tid;  // this thread's first class
    const bool active = k0 < n_cls;
    const int k_first = c0, k_last = min(c0 + S::kClasses, n_cls) - 1;
    float2 sum[C * kPair], part[C * kPair];  // .x north, .y south images
#pragma unroll
    for (int i = 0; i < C * kPair; ++i)
        sum[i] = part[i] = make_float2(0.0f, 0.0f);

    for (int q0 = rg.x; q0 <= rg.y; q0 += kRingChunk) {
        const int nq = min(kRingChunk, rg.y - q0 + 1);
        __syncthreads();
        if (tid < nq) sR[tid] = load_sym_ring(P, r, q0 + tid, rg, skip_belt_inputs);
        __syncthreads();
        for (int qi = 0; qi < nq; ++qi) {
            const SymRing g = sR[qi];
            if (g.hw < 0.0f) continue;
            const int L2 = g.len;
            // invariant the arithmetic relies on (the host's split construction
            // guarantees it): class integers fit in int32
            if (tid == 0 &&
                (long long)(2 * c0 + t) * L2 + 2LL * S::kClasses * L2 > 2147483647LL)
                atomicExch(err, KSC_ERR_DEVICE_BOUNDS);
            // the odd-step table, when the ring pair has one that fits
            if (g.onct > 0 && g.onct + 1 <= S::kXCap &&
                lockstep_pair<S, MIRROR>(P, g, c0, n_cls, t, L, m, st, xt, sW, sum, part))
                continue;
            // per-pair weights: the union of this thread's classes' windows
            long long num0, numx;
            int lo[C], hi[C], U0, U1, dummy;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                long long nc;
                sym_window(k0 + c, t, L, g, &nc, &lo[c], &hi[c]);
                if (c == 0) num0 = nc;
            }
            sym_window(k_first, t, L, g, &numx, &U0, &dummy);
            sym_window(k_last, t, L, g, &numx, &dummy, &U1);
            const int wa = lo[0], wb = hi[C - 1];
            for (int s0 = U0 & ~3; s0 <= U1; s0 += kSpan) {
                // positions this segment needs (the union ends at U1)
                const int span = min(kSpan, ((U1 - s0 + 1) + 3) & ~3);
                __syncthreads();  // the previous segment is consumed
                stage<S, MIRROR>(g, m, st, s0, span);
                __syncthreads();
                if (!active) continue;
                const int a = max(wa, s0), b = min(wb, s0 + span - 1);
                if (a > b) continue;
                // (classes without a reflection partner accumulate the reflected
                // images too; those sums are never written)
                if (g.small)
                    acc_pairs<S, 1>(P, g, st, s0, a, b, num0, L, lo, hi, sum, part);
                else
                    acc_pairs<S, 0>(P, g, st, s0, a, b, num0, L, lo, hi, sum, part);
            }
        }
    }
    // the sums with the low parts their last steps carried
#pragma unroll
    for (int i = 0; i < C * kPair; ++i) sum[i] = __fadd2_rn(sum[i], part[i]);
    const int rs = P.nrings - 1 - r;
    const int start_s = P.d_rings[rs].start;
    const bool wn = r >= band_lo && r <= band_hi;
    const bool ws = MIRROR && rs >= band_lo && rs <= band_hi;
#pragma unroll
    for (int cl = 0; cl < C; ++cl) {
        const int k = k0 + cl;
        if (k >= n_cls) break;
        // reflection partner of k; none when it is k itself up to a quarter turn
        const int kb = Q - k - t;
        const bool refl = kb != k && kb != Q;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c == 1 && !refl) break;
            const int kk = c ? kb : k;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int kq = kk + qq * Q;
                const float vn = sum[cl * kPair + 4 * c + qq].x * P.domega;
                if (wn) {
                    if (add) o[R.start + kq] += vn;
                    else o[R.start + kq] = vn;
                }
                if constexpr (MIRROR) {
                    const float vs = sum[cl * kPair + 4 * c + qq].y * P.domega;
                    if (ws) {
                        if (add) o[start_s + kq] += vs;
                        else o[start_s + kq] = vs;
                    }
                }
            }
        }
    }
}

// One work item: classes [k0, k0 + S::kClasses) of northern ring `ring` of one map.
template <class S>
__device__ __forceinline__ void sym_dispatch(const ConvPlan &P, int ring, int k0, int belt_split,
                                             int band_lo, int band_hi, const float *m, float *o,
                                             SymRing *sR, float *st, float4 *xt, int *sW,
                                             int *err) {
    const int eq = (P.nrings - 1) / 2;  // the equator ring, its own mirror image
    const DevRing R = P.d_rings[ring];
    const int Q = R.len / 4;
    const int n_cls = R.phase ? (Q + 1) / 2 : Q / 2 + 1;  // reflection classes
    const bool belt = ring >= P.belt_lo && ring <= P.belt_hi;
    const bool add = belt_split && belt;
    if (ring == eq)
        sym_item<S, false>(P, ring, k0, n_cls, add, add, band_lo, band_hi, m, o, sR, st, xt, sW,
                           err);
    else
        sym_item<S, true>(P, ring, k0, n_cls, add, add, band_lo, band_hi, m, o, sR, st, xt, sW,
                          err);
}

// One split; grid.y runs over maps.  CTAs claim items in list order through a
// counter per map (zero at launch), so the long items of a longest-first list
// start first and the short ones fill the tail.  (One code path for whole maps
// and latitude bands keeps their outputs bitwise equal.)
template <class S>
__global__ void __launch_bounds__(S::T, S::MINB)
conv_sym_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                const float *__restrict__ in, float *__restrict__ out, long long map_stride,
                int belt_split, int band_lo, int band_hi, int *__restrict__ counters,
                int *__restrict__ err) {
    __shared__ SymRing sR[kRingChunk];
    __shared__ int sW[4 * (S::T / 32)];  // per-warp walk extents (lockstep path)
    __shared__ __align__(16) float st[kImg * S::kStride];
    __shared__ int s_next;
    extern __shared__ float4 xt[];  // S::kXCap cells
    const float *m = in + (long long)blockIdx.y * map_stride;
    float *o = out + (long long)blockIdx.y * map_stride;
    for (;;) {
        __syncthreads();  // every thread has read the previous claim
        if (threadIdx.x == 0) s_next = atomicAdd(&counters[blockIdx.y], 1);
        __syncthreads();
        const int it = s_next;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        sym_dispatch<S>(P, w.ring, w.k0, belt_split, band_lo, band_hi, m, o, sR, st, xt, sW, err);
    }
}

// A batch of (split, map) entries: persistent CTAs claim items (entry, ring,
// first class) from a global counter in list order (longest first).
template <class S>
__global__ void __launch_bounds__(S::T, S::MINB)
conv_sym_batch_kernel(const ConvPlan *__restrict__ plans, const BatchEntry *__restrict__ entries,
                      const int4 *__restrict__ items, int n_items, int *__restrict__ counter,
                      int *__restrict__ err) {
    __shared__ SymRing sR[kRingChunk];
    __shared__ int sW[4 * (S::T / 32)];  // per-warp walk extents (lockstep path)
    __shared__ __align__(16) float st[kImg * S::kStride];
    __shared__ int s_next;
    extern __shared__ float4 xt[];  // S::kXCap cells
    for (;;) {
        __syncthreads();  // every thread has read the previous claim
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_next;
        if (it >= n_items) break;
        const int4 w = items[it];
        const BatchEntry e = entries[w.x];
        const ConvPlan &P = plans[e.plan];
        sym_dispatch<S>(P, w.y, w.z, e.belt_split, 0, P.nrings - 1, e.in, e.out, sR, st, xt, sW,
                        err);
    }
}

int sm_count_sym() {
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    return n_sm;
}

// Grid of a persistent launch; the kernel's dynamic shared memory (the table)
// is enabled on first use.
template <class K>
cudaError_t sym_grid(K kernel, int threads, size_t dyn_smem, int n_items, int per_sm_cap,
                     int *blocks) {
    cudaError_t e;
    if (dyn_smem > 0 &&
        (e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)dyn_smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem);
    if (e != cudaSuccess) return e;
    if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
    if (per_sm < 1) per_sm = 1;
    *blocks = n_items < sm_count_sym() * per_sm ? n_items : sm_count_sym() * per_sm;
    return cudaSuccess;
}

template <class S>
cudaError_t sym_launch(const ConvPlan &p, const WorkItem *d_items, int n_items,
                       const float *d_in, float *d_out, int n_maps, long long map_stride,
                       int belt_split, int band_lo, int band_hi, int *d_err, cudaStream_t st) {
    int blocks = 0;
    cudaError_t e = sym_grid(conv_sym_kernel<S>, S::T, S::kDynSmem, n_items, 0, &blocks);
    if (e != cudaSuccess) return e;
    // per-call claim counters, stream-ordered so that calls on several streams
    // may overlap
    int *ctr = nullptr;
    const size_t bytes = sizeof(int) * (size_t)n_maps;
    if ((e = cudaMallocAsync(&ctr, bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctr, 0, bytes, st)) == cudaSuccess) {
        dim3 grid(blocks, n_maps);
        conv_sym_kernel<S><<<grid, S::T, S::kDynSmem, st>>>(p, d_items, n_items, d_in, d_out,
                                                           map_stride, belt_split, band_lo,
                                                           band_hi, ctr, d_err);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(ctr, st);
    return e != cudaSuccess ? e : f;
}

} // namespace

int sym_classes(int len, int phase) {
    const int Q = len / 4;
    return phase ? (Q + 1) / 2 : Q / 2 + 1;
}

// Single-map items: 384 classes (3 per thread) where rings are long enough for
// many of them (nside >= 2048), else 128 (smaller items balance a launch better).
int sym_chunk(int nside) { return nside >= 2048 ? ShapeC3::kClasses : ShapeWide::kClasses; }

cudaError_t launch_conv_sym(const ConvPlan &p, const WorkItem *d_items, int n_items,
                            const float *d_in, float *d_out, int n_maps, long long map_stride,
                            int belt_split, int band_lo, int band_hi, int *d_err,
                            cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    if (sym_chunk(p.nside) == ShapeC3::kClasses)
        return sym_launch<ShapeC3>(p, d_items, n_items, d_in, d_out, n_maps, map_stride,
                                   belt_split, band_lo, band_hi, d_err, st);
    return sym_launch<ShapeWide>(p, d_items, n_items, d_in, d_out, n_maps, map_stride,
                                 belt_split, band_lo, band_hi, d_err, st);
}

int sym_variants() { return 3; }

int sym_variant_chunk(int variant) {
    return variant == 0 ? ShapeC3::kClasses
                        : (variant == 1 ? ShapeSmall::kClasses : ShapeWide::kClasses);
}

template <class S>
cudaError_t sym_batch_launch(const ConvPlan *d_plans, const BatchEntry *d_entries,
                             const int4 *d_items, int n_items, int per_sm_cap, int *d_counter,
                             int *d_err, cudaStream_t st) {
    int blocks = 0;
    cudaError_t e =
        sym_grid(conv_sym_batch_kernel<S>, S::T, S::kDynSmem, n_items, per_sm_cap, &blocks);
    if (e != cudaSuccess) return e;
    conv_sym_batch_kernel<S><<<blocks, S::T, S::kDynSmem, st>>>(d_plans, d_entries, d_items,
                                                                n_items, d_counter, d_err);
    return cudaGetLastError();
}

cudaError_t launch_conv_sym_batch(int variant, const ConvPlan *d_plans,
                                  const BatchEntry *d_entries, const int4 *d_items, int n_items,
                                  int per_sm_cap, int *d_counter, int *d_err, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (variant == 2)
        return sym_batch_launch<ShapeWide>(d_plans, d_entries, d_items, n_items, per_sm_cap,
                                           d_counter, d_err, st);
    if (variant == 1)
        return sym_batch_launch<ShapeSmall>(d_plans, d_entries, d_items, n_items, per_sm_cap,
                                            d_counter, d_err, st);
    return sym_batch_launch<ShapeC3>(d_plans, d_entries, d_items, n_items, per_sm_cap,
                                     d_counter, d_err, st);
}

} // namespace ksc
