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
// its own mirror image).  Per input ring the CTA stages, for the union of its
// threads' windows, the sixteen image sequences m[image(k')] in shared memory
// so that every image of input position k' sits at the same offset; each
// thread then walks its window four positions at a time: four independent
// kernel weights, then one 16-byte shared load per image feeding four FFMAs.
// A weight depends on the pixel pair only through the exact integer
// N = (2k + t) L' - (2k' + t') L, dphi / 2 = N pi / (2 L L').  Per input ring
// the CTA first builds the ring pair's weight table in dphi in shared memory
// (cubic cells, each from the double-float chord and the K_r table at its two
// ends, ksc_sym.cuh); a weight is then one cell lookup and three FMAs.  Ring
// pairs without a table (whole-ring windows, or more cells than a CTA holds)
// evaluate the double-float chord and the K_r table per pair (ksc_device.cuh).
// FP32 partial sums over 32 positions are Kahan-folded into the totals.
//
// Paired lanes (tile variant 2): two adjacent lanes own one class.  Each
// evaluates two of every four kernel weights, the pair swaps them with one
// shuffle, and each lane accumulates one hemisphere (eight images).  The work
// per class is the same; the accumulators per thread halve, so more warps fit
// on an SM to hide the latency of the double-float chains.
#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_sym.cuh"

namespace ksc {
namespace {

constexpr int kRingChunk = 32;  // ring-pair constants staged per pass
constexpr int kImg = 16;        // 4 rotations x {north, south} x {direct, reflected}
// Tile shape: T threads, LANES lanes per reflection class (1, or 2 for paired
// lanes), SPAN staged input positions per segment (each image row padded by 4
// floats), MINB resident CTAs per SM the register budget is set for.
// XCAP: x-table cells held in dynamic shared memory (0: weights evaluated
// directly for every pair).
template <int T_, int LANES_, int SPAN_, int MINB_, int XCAP_> struct SymShape {
    static constexpr int T = T_, LANES = LANES_, kSpan = SPAN_, MINB = MINB_;
    static constexpr int kStride = SPAN_ + 4;
    static constexpr int kClasses = T_ / LANES_;      // classes per item
    static constexpr int kImgT = kImg / LANES_;       // images per thread
    static constexpr int kXCap = XCAP_;
    static constexpr size_t kDynSmem = sizeof(float4) * (size_t)XCAP_;
};
using ShapeFull = SymShape<128, 1, 384, 4, kXCap>;  // variant 0
using ShapeHalf = SymShape<64, 1, 256, 6, 0>;       // variant 1
using ShapePair = SymShape<128, 2, 384, 5, 0>;      // variant 2

__device__ __forceinline__ void kahan(float *sum, float *comp, float v) {
    const float y = v - *comp;
    const float tt = *sum + y;
    *comp = (tt - *sum) - y;
    *sum = tt;
}

// Row of thread image i in the staged block: images are ordered
// [direct q0..q3 | mirror direct q0..q3 | reflected q0..q3 | mirror reflected];
// with paired lanes, lane h (0 north, 1 south) takes rows 4h..4h+3 and 8+4h..
__device__ __forceinline__ int img_row(int i, int lanes, int h) {
    if (lanes == 1) return i;
    return i < 4 ? 4 * h + i : 8 + 4 * h + (i - 4);
}

// The four kernel weights of quad kq (positions kq .. kq + 3; zero outside
// [a, b] and beyond the cut).  With paired lanes each lane evaluates two and
// the pair swaps them.  Straight-line code: the evaluations interleave.
// MODE 0: double-float chord with the general sine; 1: with the small-angle
// sine; 2: the ring pair's x table (partial windows only: every position
// outside [a, b] then lies beyond the cut, so the cut test alone zeroes it).
template <class S, int MODE>
__device__ __forceinline__ float4 quad_weights(const ConvPlan &P, const SymRing &g,
                                               const float4 *xt, int kq, int a, int b,
                                               long long num, int L, int h, unsigned pair_mask) {
    const float N0 = (float)(num - 2LL * kq * L);  // exact integer below 2^24
    const float step = (float)(2 * L);
    float w[4];
    constexpr int NE = 4 / S::LANES;  // weights evaluated by this lane
#pragma unroll
    for (int ee = 0; ee < NE; ++ee) {
        const int e = S::LANES == 2 ? 2 * h + ee : ee;
        const float Nf = N0 - (float)e * step;
        if constexpr (MODE == 2)
            w[ee] = xtab_weight(xt, g, Nf);
        else
            w[ee] = sym_weight<MODE == 1>(P, g, Nf, kq + e, a, b);
    }
    if constexpr (S::LANES == 2) {  // swap halves with the partner lane
        const float o0 = __shfl_xor_sync(pair_mask, w[0], 1);
        const float o1 = __shfl_xor_sync(pair_mask, w[1], 1);
        if (h == 0) { w[2] = o0; w[3] = o1; }
        else { w[2] = w[0]; w[3] = w[1]; w[0] = o0; w[1] = o1; }
    }
    return make_float4(w[0], w[1], w[2], w[3]);
}

// Positions a..b of one staged segment (starting at s0) for one thread.  The
// loop is software-pipelined: the weights of the next quad (table lookups, or
// double-float chains) are evaluated while the current quad's weights feed the
// FFMAs.
template <class S, bool MIRROR, int MODE>
__device__ __forceinline__ void accumulate(const ConvPlan &P, const SymRing &g, const float4 *xt,
                                           const float *st, int s0, int a, int b, long long num,
                                           int L, float *sum, float *comp) {
    constexpr int kStride = S::kStride, NI = S::kImgT;
    const int h = S::LANES == 2 ? (threadIdx.x & 1) : 0;
    const unsigned pair_mask = 3u << ((threadIdx.x & 31) & ~1);
    const bool idle = S::LANES == 2 && !MIRROR && h == 1;  // no south images on the equator
    float part[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) part[i] = 0.0f;
    int nq = 0;
    int kq = s0 + ((a - s0) & ~3);
    if (kq > b) return;
    float4 wc = quad_weights<S, MODE>(P, g, xt, kq, a, b, num, L, h, pair_mask);
    for (; kq <= b; kq += 4) {
        // next quad's weights (past b they are zero and unused)
        const float4 wn = quad_weights<S, MODE>(P, g, xt, kq + 4, a, b, num, L, h, pair_mask);
        const int j = kq - s0;
        if (!idle) {
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                const int img = img_row(i, S::LANES, h);
                if (S::LANES == 1 && !MIRROR && (img & 4)) continue;
                const float4 v = *reinterpret_cast<const float4 *>(st + img * kStride + j);
                float p = part[i];
                p = fmaf(wc.x, v.x, p);
                p = fmaf(wc.y, v.y, p);
                p = fmaf(wc.z, v.z, p);
                p = fmaf(wc.w, v.w, p);
                part[i] = p;
            }
        }
        wc = wn;
        if (++nq == 8) {  // fold every 32 positions
            nq = 0;
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                kahan(&sum[i], &comp[i], part[i]);
                part[i] = 0.0f;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) kahan(&sum[i], &comp[i], part[i]);
}

template <class S, bool MIRROR>
__device__ __forceinline__ void sym_item(const ConvPlan &P, int r, int c0, int n_cls,
                                         bool skip_belt_inputs, bool add, int band_lo,
                                         int band_hi, const float *__restrict__ m,
                                         float *__restrict__ o, SymRing *sR, float *st,
                                         float4 *xt) {
    constexpr int T = S::T, kSpan = S::kSpan, kStride = S::kStride, NI = S::kImgT;
    const int tid = threadIdx.x;
    const int h = S::LANES == 2 ? (tid & 1) : 0;  // paired lanes: hemisphere
    const DevRing R = P.d_rings[r];
    const int L = R.len, Q = L / 4, t = R.phase;
    const int2 rg = P.d_range[r];
    const int k = c0 + tid / S::LANES;
    const bool active = k < n_cls;
    const int k_first = c0, k_last = min(c0 + S::kClasses, n_cls) - 1;
    // reflection partner of k; none when it is k itself up to a quarter turn
    const int kb = Q - k - t;
    const bool refl = kb != k && kb != Q;
    float sum[NI], comp[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) sum[i] = comp[i] = 0.0f;

    for (int q0 = rg.x; q0 <= rg.y; q0 += kRingChunk) {
        const int nq = min(kRingChunk, rg.y - q0 + 1);
        __syncthreads();
        if (tid < nq) sR[tid] = load_sym_ring(P, r, q0 + tid, rg, skip_belt_inputs);
        __syncthreads();
        for (int qi = 0; qi < nq; ++qi) {
            const SymRing g = sR[qi];
            if (g.hw < 0.0f) continue;
            const int L2 = g.len, Q2 = L2 / 4;
            long long num, numx;
            int klo, khi, U0, U1, dummy;
            sym_window(k, t, L, g, &num, &klo, &khi);
            sym_window(k_first, t, L, g, &numx, &U0, &dummy);
            sym_window(k_last, t, L, g, &numx, &dummy, &U1);
            const bool use_xt = S::kXCap > 0 && g.ncell > 0 && g.ncell <= S::kXCap;
            if (use_xt) {  // (the segment's first barrier publishes the table)
                __syncthreads();  // the previous ring pair's lookups are done
                xtab_build<S::T>(P, g, xt);
            }
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
                const int a = max(klo, s0), b = min(khi, s0 + kSpan - 1);
                if (a > b) continue;
                // (classes without a reflection partner accumulate the reflected
                // images too; those sums are never written)
                if (S::kXCap > 0 && use_xt)
                    accumulate<S, MIRROR, 2>(P, g, xt, st, s0, a, b, num, L, sum, comp);
                else if (g.small)
                    accumulate<S, MIRROR, 1>(P, g, xt, st, s0, a, b, num, L, sum, comp);
                else
                    accumulate<S, MIRROR, 0>(P, g, xt, st, s0, a, b, num, L, sum, comp);
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
                if (S::LANES == 1) {
                    const float vn = sum[8 * c + qq] * P.domega;
                    if (wn) {
                        if (add) o[R.start + kq] += vn;
                        else o[R.start + kq] = vn;
                    }
                    if constexpr (MIRROR) {
                        const float vs = sum[8 * c + 4 + qq] * P.domega;
                        if (ws) {
                            if (add) o[start_s + kq] += vs;
                            else o[start_s + kq] = vs;
                        }
                    }
                } else {  // lane h writes its hemisphere
                    const float v = sum[4 * c + qq] * P.domega;
                    const bool wr = h == 0 ? wn : ws;
                    const int base = h == 0 ? R.start : start_s;
                    if (wr) {
                        if (add) o[base + kq] += v;
                        else o[base + kq] = v;
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
                                             SymRing *sR, float *st, float4 *xt) {
    const int eq = (P.nrings - 1) / 2;  // the equator ring, its own mirror image
    const DevRing R = P.d_rings[ring];
    const int Q = R.len / 4;
    const int n_cls = R.phase ? (Q + 1) / 2 : Q / 2 + 1;  // reflection classes
    const bool belt = ring >= P.belt_lo && ring <= P.belt_hi;
    const bool add = belt_split && belt;
    if (ring == eq)
        sym_item<S, false>(P, ring, k0, n_cls, add, add, band_lo, band_hi, m, o, sR, st, xt);
    else
        sym_item<S, true>(P, ring, k0, n_cls, add, add, band_lo, band_hi, m, o, sR, st, xt);
}

// One split; grid.y runs over maps.  CTAs claim items in list order through a
// counter per map (zero at launch), so the long items of a longest-first list
// start first and the short ones fill the tail.  (One code path for whole maps
// and latitude bands keeps their outputs bitwise equal.)
template <class S>
__global__ void __launch_bounds__(S::T, S::MINB)
conv_sym_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                const float *__restrict__ in, float *__restrict__ out, long long map_stride,
                int belt_split, int band_lo, int band_hi, int *__restrict__ counters) {
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
        sym_dispatch<S>(P, w.ring, w.k0, belt_split, band_lo, band_hi, m, o, sR, st, xt);
    }
}

// A batch of (split, map) entries: persistent CTAs claim items (entry, ring,
// first class) from a global counter in list order (longest first).
template <class S>
__global__ void __launch_bounds__(S::T, S::MINB)
conv_sym_batch_kernel(const ConvPlan *__restrict__ plans, const BatchEntry *__restrict__ entries,
                      const int4 *__restrict__ items, int n_items, int *__restrict__ counter) {
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
        sym_dispatch<S>(P, w.y, w.z, e.belt_split, 0, P.nrings - 1, e.in, e.out, sR, st, xt);
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

// Grid of a persistent launch; the kernel's dynamic shared memory (the x table)
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

} // namespace

int sym_classes(int len, int phase) {
    const int Q = len / 4;
    return phase ? (Q + 1) / 2 : Q / 2 + 1;
}

cudaError_t launch_conv_sym(const ConvPlan &p, const WorkItem *d_items, int n_items,
                            const float *d_in, float *d_out, int n_maps, long long map_stride,
                            int belt_split, int band_lo, int band_hi, cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    using S = ShapeFull;
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
                                                           band_hi, ctr);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(ctr, st);
    return e != cudaSuccess ? e : f;
}

int sym_chunk() { return ShapeFull::kClasses; }

int sym_variants() { return 3; }

int sym_variant_chunk(int variant) {
    return variant == 2 ? ShapePair::kClasses
                        : (variant == 1 ? ShapeHalf::kClasses : ShapeFull::kClasses);
}

template <class S>
cudaError_t sym_batch_launch(const ConvPlan *d_plans, const BatchEntry *d_entries,
                             const int4 *d_items, int n_items, int per_sm_cap, int *d_counter,
                             cudaStream_t st) {
    int blocks = 0;
    cudaError_t e =
        sym_grid(conv_sym_batch_kernel<S>, S::T, S::kDynSmem, n_items, per_sm_cap, &blocks);
    if (e != cudaSuccess) return e;
    conv_sym_batch_kernel<S><<<blocks, S::T, S::kDynSmem, st>>>(d_plans, d_entries, d_items,
                                                                n_items, d_counter);
    return cudaGetLastError();
}

cudaError_t launch_conv_sym_batch(int variant, const ConvPlan *d_plans,
                                  const BatchEntry *d_entries, const int4 *d_items, int n_items,
                                  int per_sm_cap, int *d_counter, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (variant == 2)
        return sym_batch_launch<ShapePair>(d_plans, d_entries, d_items, n_items, per_sm_cap,
                                           d_counter, st);
    if (variant == 1)
        return sym_batch_launch<ShapeHalf>(d_plans, d_entries, d_items, n_items, per_sm_cap,
                                           d_counter, st);
    return sym_batch_launch<ShapeFull>(d_plans, d_entries, d_items, n_items, per_sm_cap,
                                       d_counter, st);
}

} // namespace ksc
