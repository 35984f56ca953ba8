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
// memory so that every image of input position k' sits at the same offset; each
// thread then walks the union of its classes' windows four positions at a time:
// 4 C kernel weights, then one 16-byte shared load per image feeding 4 C FFMAs.
// The sixteen images of a position are loaded once for the C classes: shared-
// memory bandwidth to the lanes (a 16-byte load by a warp costs four wavefronts
// whatever its addresses) is what bounds this gather, and C classes per thread
// divide the image traffic per pixel pair by C.
//
// A weight depends on the pixel pair only through the exact integer
// N = (2k + t) L' - (2k' + t') L (dphi / 2 = N pi / (2 L L')).  Per input ring
// the CTA first builds the ring pair's weight table in |N| in shared memory
// (cubic cells of 2^shift integers whose last cell ends exactly at the cut,
// followed by a zero cell, ksc_sym.cuh); a weight is then a table position
// p = min(|N| + off, nct 2^shift) 2^-shift (exact), its cell floor(p) and offset
// p - floor(p) (exact), one 16-byte cell load and three FMAs, and it is exactly
// zero beyond the cut with no test.  Ring pairs without a table (whole-ring
// windows, or more cells than a CTA holds) evaluate the double-float chord and
// the K_r table per pair (ksc_device.cuh).  FP32 partial sums over 64 positions
// are Kahan-folded into the totals.
#include <cstdint>

#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_sym.cuh"

namespace ksc {
namespace {

constexpr int kRingChunk = 32;  // ring-pair constants staged per pass
constexpr int kImg = 16;        // 4 rotations x {north, south} x {direct, reflected}
constexpr int kFold = 16;       // quads per FP32 partial sum (64 positions)
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

__device__ __forceinline__ void kahan(float *sum, float *comp, float v) {
    const float y = v - *comp;
    const float tt = *sum + y;
    *comp = (tt - *sum) - y;
    *sum = tt;
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

// Sixteen (or, on the equator, eight) images of one quad of positions for the C
// classes of a thread: one 16-byte shared load per image, 4 C FFMAs.
template <class S, bool MIRROR>
__device__ __forceinline__ void fma_quad(const float *st, int j, const float4 *w, float *part) {
#pragma unroll
    for (int i = 0; i < kImg; ++i) {
        if (!MIRROR && (i & 4)) continue;
        const float4 v = *reinterpret_cast<const float4 *>(st + i * S::kStride + j);
#pragma unroll
        for (int c = 0; c < S::C; ++c) {
            float p = part[c * kImg + i];
            p = fmaf(w[c].x, v.x, p);
            p = fmaf(w[c].y, v.y, p);
            p = fmaf(w[c].z, v.z, p);
            p = fmaf(w[c].w, v.w, p);
            part[c * kImg + i] = p;
        }
    }
}

template <class S>
__device__ __forceinline__ void fold(float *sum, float *comp, float *part) {
#pragma unroll
    for (int i = 0; i < S::C * kImg; ++i) {
        kahan(&sum[i], &comp[i], part[i]);
        part[i] = 0.0f;
    }
}

// Constants of the table path for one ring pair: table positions are
// p = min(|N| + off, nct 2^shift) 2^-shift.
struct TabPos {
    float inv, offS, ncf;  // 2^-shift, off 2^-shift, nct
    float step, dcls;      // per position (2 L) and per class (2 L') in table units
};

// The four weights of the quad at table position tp (class c, first position).
__device__ __forceinline__ float4 tab_quad(const float4 *xt, const TabPos &x, float tp) {
    float4 w;
    w.x = xtab_at(xt, fminf(fabsf(tp) + x.offS, x.ncf));
    w.y = xtab_at(xt, fminf(fabsf(tp - x.step) + x.offS, x.ncf));
    w.z = xtab_at(xt, fminf(fabsf(fmaf(-2.0f, x.step, tp)) + x.offS, x.ncf));
    w.w = xtab_at(xt, fminf(fabsf(fmaf(-3.0f, x.step, tp)) + x.offS, x.ncf));
    return w;
}

// Table path.  Positions a..b of one staged segment (s0: its first position):
// the union of the thread's classes' windows within the cut.  Every weight
// beyond a class's cut is exactly zero (the table's zero cell), so no position
// needs a mask.  The loop is software-pipelined: the next quad's weights are
// looked up while the current quad's FFMAs run.
template <class S, bool MIRROR>
__device__ __forceinline__ void acc_table(const float4 *xt, const TabPos &x, const float *st,
                                          int s0, int a, int b, int num, int L, float *sum,
                                          float *comp, float *part) {
    constexpr int C = S::C;
    int kq = s0 + ((a - s0) & ~3);
    // exact: the thread's positions lie within a few of every class's window, where
    // |N| < 2^24
    float tp = (float)(num - 2 * L * kq) * x.inv;  // class 0 at the first quad
    float4 wc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) wc[c] = tab_quad(xt, x, fmaf((float)c, x.dcls, tp));
    int nq = 0;
    for (; kq + 4 <= b; kq += 4) {
        tp = fmaf(-4.0f, x.step, tp);
        float4 wn[C];
#pragma unroll
        for (int c = 0; c < C; ++c) wn[c] = tab_quad(xt, x, fmaf((float)c, x.dcls, tp));
        fma_quad<S, MIRROR>(st, kq - s0, wc, part);
#pragma unroll
        for (int c = 0; c < C; ++c) wc[c] = wn[c];
        if (++nq == kFold) {
            nq = 0;
            fold<S>(sum, comp, part);
        }
    }
    fma_quad<S, MIRROR>(st, kq - s0, wc, part);  // the last quad (kq <= b < kq + 4)
    fold<S>(sum, comp, part);
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
template <class S, bool MIRROR, int MODE>
__device__ __forceinline__ void acc_pairs(const ConvPlan &P, const SymRing &g, const float *st,
                                          int s0, int a, int b, long long num0, int L,
                                          const int *lo, const int *hi, float *sum, float *comp,
                                          float *part) {
    constexpr int C = S::C;
    int nq = 0;
    for (int kq = s0 + ((a - s0) & ~3); kq <= b; kq += 4) {
        // (rare: one class at a time, each loading the images again)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float4 w = quad_weights<MODE>(P, g, kq, lo[c], hi[c], num0 + 2LL * c * g.len, L);
#pragma unroll
            for (int i = 0; i < kImg; ++i) {
                if (!MIRROR && (i & 4)) continue;
                const float4 v = *reinterpret_cast<const float4 *>(st + i * S::kStride + kq - s0);
                float pp = part[c * kImg + i];
                pp = fmaf(w.x, v.x, pp);
                pp = fmaf(w.y, v.y, pp);
                pp = fmaf(w.z, v.z, pp);
                pp = fmaf(w.w, v.w, pp);
                part[c * kImg + i] = pp;
            }
        }
        if (++nq == kFold) {
            nq = 0;
            fold<S>(sum, comp, part);
        }
    }
    fold<S>(sum, comp, part);
}

template <class S, bool MIRROR>
__device__ __forceinline__ void sym_item(const ConvPlan &P, int r, int c0, int n_cls,
                                         bool skip_belt_inputs, bool add, int band_lo,
                                         int band_hi, const float *__restrict__ m,
                                         float *__restrict__ o, SymRing *sR, float *st,
                                         float4 *xt, int *__restrict__ err) {
    constexpr int T = S::T, C = S::C, kSpan = S::kSpan, kStride = S::kStride;
    const int tid = threadIdx.x;
    const DevRing R = P.d_rings[r];
    const int L = R.len, Q = L / 4, t = R.phase;
    const int2 rg = P.d_range[r];
    const int k0 = c0 + C * tid;  // this thread's first class
    const bool active = k0 < n_cls;
    const int k_first = c0, k_last = min(c0 + S::kClasses, n_cls) - 1;
    float sum[C * kImg], comp[C * kImg], part[C * kImg];
#pragma unroll
    for (int i = 0; i < C * kImg; ++i) sum[i] = comp[i] = part[i] = 0.0f;

    for (int q0 = rg.x; q0 <= rg.y; q0 += kRingChunk) {
        const int nq = min(kRingChunk, rg.y - q0 + 1);
        __syncthreads();
        if (tid < nq) sR[tid] = load_sym_ring(P, r, q0 + tid, rg, skip_belt_inputs);
        __syncthreads();
        for (int qi = 0; qi < nq; ++qi) {
            const SymRing g = sR[qi];
            if (g.hw < 0.0f) continue;
            const int L2 = g.len, Q2 = L2 / 4;
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
            // table with its last cell ending at the cut (plus one zero cell)
            const int off = (-(g.ncut + 1)) & ((1 << g.shift) - 1);
            const int nct = (g.ncut + 1 + off) >> g.shift;
            const bool use_xt = g.ncell > 0 && nct + 1 <= S::kXCap;
            // the union of this thread's classes' windows (within the cut for tables)
            int wa = lo[0], wb = hi[C - 1];
            if (use_xt) {
                wa = max(wa, ceil_div((int)num0 - g.ncut, 2 * L));
                wb = min(wb, floor_div((int)(num0 + 2LL * (C - 1) * L2) + g.ncut, 2 * L));
                __syncthreads();  // the previous ring pair's lookups are done
                xtab_build_cut<S::T>(P, g, xt, off, nct);  // (published by the next barrier)
            }
            const TabPos x{g.inv, (float)off * g.inv, (float)nct, (float)(2 * L) * g.inv,
                           (float)(2 * L2) * g.inv};
            // invariants the arithmetic relies on (the host's split construction
            // guarantees them): class integers fit in int32, and table positions within
            // a few positions of the cut stay exact in FP32
            if (tid == 0 && (num0 + 2LL * S::kClasses * L2 > 2147483647LL ||
                             (use_xt && (long long)g.ncut + 32LL * L >= (1LL << 24))))
                atomicExch(err, KSC_ERR_DEVICE_BOUNDS);
            for (int s0 = U0 & ~3; s0 <= U1; s0 += kSpan) {
                // positions this segment needs (the union ends at U1)
                const int span = min(kSpan, ((U1 - s0 + 1) + 3) & ~3);
                __syncthreads();  // the previous segment is consumed
                for (int j = tid; j < span; j += T) {
                    const int kp = s0 + j;
                    const int idx = sym_pmod(kp, L2);
                    const int idr = sym_pmod(Q2 - kp - g.phase, L2);
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        int ia = idx + qq * Q2;
                        if (ia >= L2) ia -= L2;
                        int ib = idr + qq * Q2;
                        if (ib >= L2) ib -= L2;
                        st[qq * kStride + j] = __ldg(m + g.start + ia);
                        st[(8 + qq) * kStride + j] = __ldg(m + g.start + ib);
                        if constexpr (MIRROR) {
                            st[(4 + qq) * kStride + j] = __ldg(m + g.start_m + ia);
                            st[(12 + qq) * kStride + j] = __ldg(m + g.start_m + ib);
                        }
                    }
                }
                __syncthreads();
                if (!active) continue;
                const int a = max(wa, s0), b = min(wb, s0 + span - 1);
                if (a > b) continue;
                // (classes without a reflection partner accumulate the reflected
                // images too; those sums are never written)
                if (use_xt)
                    acc_table<S, MIRROR>(xt, x, st, s0, a, b, (int)num0, L, sum, comp, part);
                else if (g.small)
                    acc_pairs<S, MIRROR, 1>(P, g, st, s0, a, b, num0, L, lo, hi, sum, comp, part);
                else
                    acc_pairs<S, MIRROR, 0>(P, g, st, s0, a, b, num0, L, lo, hi, sum, comp, part);
            }
        }
    }
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
                const float vn = sum[cl * kImg + 8 * c + qq] * P.domega;
                if (wn) {
                    if (add) o[R.start + kq] += vn;
                    else o[R.start + kq] = vn;
                }
                if constexpr (MIRROR) {
                    const float vs = sum[cl * kImg + 8 * c + 4 + qq] * P.domega;
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
                                             SymRing *sR, float *st, float4 *xt, int *err) {
    const int eq = (P.nrings - 1) / 2;  // the equator ring, its own mirror image
    const DevRing R = P.d_rings[ring];
    const int Q = R.len / 4;
    const int n_cls = R.phase ? (Q + 1) / 2 : Q / 2 + 1;  // reflection classes
    const bool belt = ring >= P.belt_lo && ring <= P.belt_hi;
    const bool add = belt_split && belt;
    if (ring == eq)
        sym_item<S, false>(P, ring, k0, n_cls, add, add, band_lo, band_hi, m, o, sR, st, xt, err);
    else
        sym_item<S, true>(P, ring, k0, n_cls, add, add, band_lo, band_hi, m, o, sR, st, xt, err);
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
        sym_dispatch<S>(P, w.ring, w.k0, belt_split, band_lo, band_hi, m, o, sR, st, xt, err);
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
        sym_dispatch<S>(P, w.y, w.z, e.belt_split, 0, P.nrings - 1, e.in, e.out, sR, st, xt,
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
