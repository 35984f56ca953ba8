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
// One thread owns one reflection class {k, kb} of first-quarter positions of
// a northern ring (a class of one when kb coincides with k up to a quarter
// turn) and produces all its images (no mirror on the equator ring, which is
// its own mirror image).  The chord and table position are computed in
// double-float from FP64 ring-pair constants and the exact integer
// N = (2k + t) L' - (2k' + t') L with dphi / 2 = N pi / (2 L L')
// (ksc_device.cuh); K_r comes from the cubic Hermite table through the L1
// cache.  Each input ring's FP32 partial sums are Kahan-folded into totals.
#include "ksc_device.cuh"
#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr int kThreads = 128;
constexpr int kRingChunk = 64;


struct SymRing {  // shared-memory constants of one (output ring, input ring) pair
    DF A, B, c;
    float hw;
    int len, start, start_m, phase;
};

template <bool MIRROR>
__device__ __forceinline__ void sym_item(const ConvPlan &P, int r, int k, bool active,
                                         bool skip_belt_inputs, bool add, int band_lo,
                                         int band_hi, const float *__restrict__ m,
                                         float *__restrict__ o, SymRing *sR) {
    const int tid = threadIdx.x;
    const DevRing R = P.d_rings[r];
    const int L = R.len, Q = L / 4, t = R.phase;
    const int2 rg = P.d_range[r];
    // reflection partner of k; none when it is k itself up to a quarter turn
    const int kb = Q - k - t;
    const bool refl = kb != k && kb != Q;
    constexpr int NI = MIRROR ? 8 : 4;  // images per class member
    float sum[2 * NI], comp[2 * NI];
#pragma unroll
    for (int i = 0; i < 2 * NI; ++i) sum[i] = comp[i] = 0.0f;

    for (int q0 = rg.x; q0 <= rg.y; q0 += kRingChunk) {
        const int nq = min(kRingChunk, rg.y - q0 + 1);
        __syncthreads();
        if (tid < nq) {
            const int q = q0 + tid;
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
            sR[tid] = g;
        }
        __syncthreads();
        if (!active) continue;
        for (int qi = 0; qi < nq; ++qi) {
            const SymRing g = sR[qi];
            if (g.hw < 0.0f) continue;
            const int L2 = g.len, Q2 = L2 / 4;
            const long long num = (long long)(2 * k + t) * L2 - (long long)g.phase * L;
            const float kc = (float)num / (float)(2 * L);
            int klo = (int)floorf(kc - g.hw), khi = (int)ceilf(kc + g.hw);
            if (2.0f * g.hw + 1.0f >= (float)L2 || khi - klo + 1 >= L2) {
                klo = (int)floorf(kc) - L2 / 2;
                khi = klo + L2 - 1;
            }
            float Nf = (float)(num - 2LL * klo * L);  // exact integer below 2^24
            const float step = (float)(2 * L);
            int idx = klo % L2;               // k' mod L2
            if (idx < 0) idx += L2;
            int idb = (Q2 - klo - g.phase) % L2;  // (Q2 - k' - t') mod L2
            if (idb < 0) idb += L2;
            const float *mn = m + g.start;
            const float *ms = m + g.start_m;
            // blocks of 32 window steps: FP32 partial sums, Kahan-folded into
            // the totals after each block
            for (int kb0 = klo; kb0 <= khi; kb0 += 32) {
                const int kend = min(kb0 + 31, khi);
                float part[2 * NI];
#pragma unroll
                for (int i = 0; i < 2 * NI; ++i) part[i] = 0.0f;
                for (int kk = kb0; kk <= kend; ++kk) {
                    const float xh = Nf * g.c.h;
                    const float xl = fmaf(Nf, g.c.h, -xh) + Nf * g.c.l;
                    int ti;
                    float f;
                    if (chord_to_table(g.A, g.B, sin_df(xh, xl), P.nint2, P.n_int, &ti, &f)) {
                        const float w = hermite(__ldg(&P.d_tab[ti]), f);
                        int j = idx, jb = idb;
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) {
                            part[qq] = fmaf(w, __ldg(mn + j), part[qq]);
                            if constexpr (MIRROR)
                                part[4 + qq] = fmaf(w, __ldg(ms + j), part[4 + qq]);
                            if (refl) {
                                part[NI + qq] = fmaf(w, __ldg(mn + jb), part[NI + qq]);
                                if constexpr (MIRROR)
                                    part[NI + 4 + qq] = fmaf(w, __ldg(ms + jb), part[NI + 4 + qq]);
                            }
                            j += Q2;
                            if (j >= L2) j -= L2;
                            jb += Q2;
                            if (jb >= L2) jb -= L2;
                        }
                    }
                    Nf -= step;
                    if (++idx == L2) idx = 0;
                    if (--idb < 0) idb = L2 - 1;
                }
#pragma unroll
                for (int i = 0; i < 2 * NI; ++i) {
                    const float y = part[i] - comp[i];
                    const float tt = sum[i] + y;
                    comp[i] = (tt - sum[i]) - y;
                    sum[i] = tt;
                }
            }
        }
    }
    if (active) {
        const int rs = P.nrings - 1 - r;
        const int start_s = P.d_rings[rs].start;
        const bool wn = r >= band_lo && r <= band_hi;
        const bool ws = MIRROR && rs >= band_lo && rs <= band_hi;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c == 1 && !refl) break;
            const int kk = c ? kb : k;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int kq = kk + qq * Q;
                const float vn = sum[c * NI + qq] * P.domega;
                if (wn) {
                    if (add) o[R.start + kq] += vn;
                    else o[R.start + kq] = vn;
                }
                if constexpr (MIRROR) {
                    const float vs = sum[c * NI + 4 + qq] * P.domega;
                    if (ws) {
                        if (add) o[start_s + kq] += vs;
                        else o[start_s + kq] = vs;
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads)
conv_sym_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                const float *__restrict__ in, float *__restrict__ out, long long map_stride,
                int belt_split, int band_lo, int band_hi) {
    __shared__ SymRing sR[kRingChunk];
    const float *m = in + (long long)blockIdx.y * map_stride;
    float *o = out + (long long)blockIdx.y * map_stride;
    const int eq = (P.nrings - 1) / 2;  // the equator ring, its own mirror image
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const DevRing R = P.d_rings[w.ring];
        const int Q = R.len / 4;
        const int n_cls = R.phase ? (Q + 1) / 2 : Q / 2 + 1;  // reflection classes
        const int k = w.k0 + threadIdx.x;
        const bool active = k < n_cls;
        const bool belt = w.ring >= P.belt_lo && w.ring <= P.belt_hi;
        const bool add = belt_split && belt;
        if (w.ring == eq)
            sym_item<false>(P, w.ring, k, active, add, add, band_lo, band_hi, m, o, sR);
        else
            sym_item<true>(P, w.ring, k, active, add, add, band_lo, band_hi, m, o, sR);
    }
}

} // namespace

int sym_classes(int len, int phase) {
    const int Q = len / 4;
    return phase ? (Q + 1) / 2 : Q / 2 + 1;
}

cudaError_t launch_conv_sym(const ConvPlan &p, const WorkItem *d_items, int n_items,
                            const float *d_in, float *d_out, int n_maps, long long map_stride,
                            int belt_split, int band_lo, int band_hi, cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    int per_sm = 0;
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_sym_kernel, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int blocks = n_sm * per_sm;
    if (blocks > n_items) blocks = n_items;
    dim3 grid(blocks, n_maps);
    conv_sym_kernel<<<grid, kThreads, 0, st>>>(p, d_items, n_items, d_in, d_out, map_stride,
                                               belt_split, band_lo, band_hi);
    return cudaGetLastError();
}

int sym_chunk() { return kThreads; }

} // namespace ksc
