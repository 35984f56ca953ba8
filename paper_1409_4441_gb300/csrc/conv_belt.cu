// Real-space convolution, equatorial-belt ring pairs (circulant form).
//
// In the HEALPix belt (|z| <= 2/3) every ring has L = 4 nside pixels.  For an
// output ring and an input ring of the belt, pixel k of the first and k' of
// the second are dphi apart with dphi/2 = (t - t' - 2 (k' - k)) pi / (2L), so
// the kernel weight depends on Delta = k' - k only:
//
//   out_r[k] += sum_Delta w_{r r'}[Delta] * m_{r'}[(k + Delta) mod L]
//
// (a circular correlation).  Each CTA owns a chunk of C = kU * kThreads
// consecutive output pixels of one belt ring and walks the belt input rings
// within theta_cut.  Per input ring it
//   1. issues 1-D TMA bulk copies (cp.async.bulk, mbarrier completion) of the
//      input segment m_{r'}[k0 + Delta_0 .. k0 + Delta_0 + C + nD - 1] (wrapped
//      round the ring) into the other shared-memory buffer, ahead of use;
//   2. computes the weight vector w[Delta] (chord^2 = A + B sin^2(dphi/2) from
//      FP64 ring constants, cubic Hermite table, zero outside the cut);
//   3. runs the FFMA sliding window: each thread keeps kU consecutive outputs
//      in registers; a block of kU weights and 2kU-1 inputs gives kU*kU FFMAs
//      for 2kU shared-memory loads.  kU is odd, so the kU-word stride between
//      lanes hits 32 distinct banks.
//   4. folds the FP32 ring partial sums into the totals with Kahan steps, at
//      the end of the ring pair and, where the pair's closest approach is near,
//      right after the half block that holds its largest terms.
// Every mbarrier wait is bounded; a wait that runs out raises a device error
// flag and the kernel stops work instead of hanging.
#include <algorithm>
#include <cstdint>

#include "ksc_device.cuh"
#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr int kU = 13;          // outputs per thread (odd: conflict-free strides)
constexpr int kThreads = 160;   // 5 warps
constexpr int kChunk = kU * kThreads;  // outputs per item of the single-split kernel
constexpr int kMaxWait = 1 << 22;   // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for the given phase parity; returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < kMaxWait; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Kahan step: sum + comp carries the total, v is the next partial sum.
__device__ __forceinline__ void kahan(float &sum, float &comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// One block of 2 kU steps of the sliding window, acc[u] += w[j] seg[u + j] for
// j in [j0, j0 + 2 kU), then acc into the ring partial.  On entry values
// j0 .. j0 + kU - 2 of the segment sit in R0[0 .. kU - 2]; on exit values
// j0 + 2 kU .. j0 + 3 kU - 2 do.
// With MID_FOLD the ring partial and the first half's steps are folded into the
// totals (sum, comp) between the two halves.
template <bool MID_FOLD>
__device__ __forceinline__ void belt_block(const float *sg, const float *wbuf, int j0,
                                           float (&R0)[2 * kU], float (&acc)[kU],
                                           float (&ring)[kU], float (&sum)[kU],
                                           float (&comp)[kU]) {
    // block A: values j0 .. j0 + 2kU - 2 live in R0[(v) % 2kU]
#pragma unroll
    for (int e = kU - 1; e < 2 * kU - 1; ++e) R0[e] = sg[j0 + e];
#pragma unroll
    for (int jj = 0; jj < kU; ++jj) {
        const float wv = wbuf[j0 + jj];
#pragma unroll
        for (int u = 0; u < kU; ++u) acc[u] = fmaf(wv, R0[u + jj], acc[u]);
    }
    if constexpr (MID_FOLD) {
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            kahan(sum[u], comp[u], ring[u] + acc[u]);
            acc[u] = ring[u] = 0.0f;
        }
    }
    // block B: values j0 + kU .. j0 + 3kU - 2 -> R0[(v - j0) % 2kU]
#pragma unroll
    for (int e = 2 * kU - 1; e < 3 * kU - 1; ++e) R0[e % (2 * kU)] = sg[j0 + e];
#pragma unroll
    for (int jj = 0; jj < kU; ++jj) {
        const float wv = wbuf[j0 + kU + jj];
#pragma unroll
        for (int u = 0; u < kU; ++u) acc[u] = fmaf(wv, R0[(kU + u + jj) % (2 * kU)], acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        ring[u] += acc[u];
        acc[u] = 0.0f;
    }
}

struct PairGeom {
    DF A, B, c1;        // (chord n_int/d_cut)^2 = A + B sin^2(x), x = (t - t' - 2 Delta) c1
    int d0;             // first Delta of the padded window
    int nd;             // padded window length (multiple of 2 kU)
    int exact_lo, exact_hi;  // Delta range that may carry weight (at most L values)
    int tdiff;          // t - t'
    bool empty;
};

// Window of a belt ring pair from its precomputed geometry.
__device__ __forceinline__ PairGeom pair_geom(const PairInfo &pi, int L, int tdiff, float c1h,
                                              float c1l) {
    PairGeom g;
    g.A = DF{pi.Ah, pi.Al};
    g.B = DF{pi.Bh, pi.Bl};
    g.c1 = DF{c1h, c1l};
    g.tdiff = tdiff;
    g.empty = pi.w < 0;
    int lo = -pi.w, hi = pi.w;
    if (hi - lo + 1 >= L) {  // whole ring: each input pixel exactly once
        lo = -(L / 2);
        hi = lo + L - 1;
    }
    g.exact_lo = lo;
    g.exact_hi = hi;
    const int n = hi - lo + 1;
    g.d0 = lo;
    g.nd = ((n + 2 * kU - 1) / (2 * kU)) * (2 * kU);
    return g;
}

// One work item: outputs [k0, k0 + T kU) of belt ring r of one map.  The
// shared buffers, barriers and their phases persist across items.  Returns
// false when a bounded wait ran out (the error flag is set and any copy still
// in flight has been waited for): the CTA must stop.
template <int T>
__device__ __forceinline__ bool belt_item(const ConvPlan &P, int r, int k0,
                                          const float *__restrict__ m, float *__restrict__ o,
                                          float *seg0, float *seg1, float *wbuf, uint64_t *bar,
                                          PairGeom *s_g, int *s_abort, uint32_t &phase0,
                                          uint32_t &phase1, int seg_cap, int *__restrict__ err) {
    constexpr int kChunkT = kU * T;
    const int tid = threadIdx.x;
    const DevRing R = P.d_rings[r];
    const int L = R.len;
    const int2 rg = P.d_range[r];
    const int q_lo = max(rg.x, P.belt_lo), q_hi = min(rg.y, P.belt_hi);
    const int kb = tid * kU;  // first output (chunk-relative) of this thread
    float sum[kU], comp[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) sum[u] = comp[u] = 0.0f;

    // issue the copy of input ring q into buffer b
    const PairInfo *pinfo = P.d_pairs + P.d_pair_base[r] - rg.x;
    auto issue = [&](int q, int b) {
        const DevRing Q = P.d_rings[q];
        PairGeom g = pair_geom(pinfo[q], L, R.phase - Q.phase, P.belt_c1h, P.belt_c1l);
        s_g[b] = g;
        if (g.empty) return;
        // ring coordinates [a, a + n), a aligned down to 4 floats
        int a = k0 + g.d0;
        int n = kChunkT + g.nd - 1;
        int a4 = a & ~3;  // floor to a multiple of 4 (also for negatives)
        n += a - a4;
        n = (n + 3) & ~3;
        if (n > seg_cap) {  // never expected: the host sized seg_cap for every pair
            atomicExch(err, KSC_ERR_DEVICE_BOUNDS);
            s_g[b].empty = true;
            return;
        }
        float *dst = b ? seg1 : seg0;
        const float *ring = m + Q.start;
        uint32_t total = 4u * (uint32_t)n;
        mbar_expect_tx(&bar[b], total);
        int pos = a4, done = 0;
        while (done < n) {
            int pm = ((pos % L) + L) % L;
            int len = min(n - done, L - pm);
            bulk_g2s(dst + done, ring + pm, 4u * (uint32_t)len, &bar[b]);
            done += len;
            pos += len;
        }
    };

    if (tid == 0 && q_lo <= q_hi) issue(q_lo, 0);
    int b = 0;
    for (int q = q_lo; q <= q_hi; ++q, b ^= 1) {
        __syncthreads();  // previous pair's buffers are free; s_g[b] visible
        if (tid == 0 && q + 1 <= q_hi) issue(q + 1, b ^ 1);
        const PairGeom g = s_g[b];
        if (g.empty) continue;
        // weights for this ring pair (zero outside the cut / exact window)
        for (int j = tid; j < g.nd; j += T) {
            const int D = g.d0 + j;
            float wv = 0.0f;
            if (D >= g.exact_lo && D <= g.exact_hi) {
                const float mf = (float)(g.tdiff - 2 * D);
                const float xh = mf * g.c1.h;
                const float xl = fmaf(mf, g.c1.h, -xh) + mf * g.c1.l;
                int ti;
                float f;
                if (chord_to_table(g.A, g.B, sin_df(xh, xl), P.nint2, P.n_int, &ti, &f))
                    wv = hermite(__ldg(&P.d_tab[ti]), f);
            }
            wbuf[j] = wv;
        }
        const bool ok = mbar_wait(&bar[b], b ? phase1 : phase0);
        if (ok) {
            if (b) phase1 ^= 1u; else phase0 ^= 1u;
        } else {
            *s_abort = 1;
        }
        __syncthreads();
        if (*s_abort) break;
        // sliding-window FFMA: acc[u] = sum_j w[j] * seg[off + kb + u + j]
        const float *sg = (b ? seg1 : seg0) + ((k0 + g.d0) - ((k0 + g.d0) & ~3)) + kb;
        float acc[kU], ring[kU];  // block (2 kU steps) and ring-pair partial sums
#pragma unroll
        for (int u = 0; u < kU; ++u) acc[u] = ring[u] = 0.0f;
        float R0[2 * kU];
#pragma unroll
        for (int e = 0; e < kU - 1; ++e) R0[e] = sg[e];
        // The largest terms of a ring pair lie at its closest approach, Delta in
        // [-2, 3] (step j = 3 - d0 the last of them).  Where that approach is within
        // an eighth of the cut, the ring partial is folded into the totals right
        // after the half block (kU steps) holding j = 3 - d0, so that the later
        // steps do not round at the size of those terms.  That block runs apart
        // from the two loops around it, which stay free of the test.
        const bool near = g.A.h < P.nint2 * (1.0f / 64.0f);
        const int jpk = 3 - g.d0;
        const int jb = near ? min(g.nd, (jpk / (2 * kU)) * (2 * kU)) : g.nd;
        int j0 = 0;
        for (; j0 < jb; j0 += 2 * kU) belt_block<false>(sg, wbuf, j0, R0, acc, ring, sum, comp);
        if (j0 < g.nd) {
            if (jpk - j0 < kU) {
                belt_block<true>(sg, wbuf, j0, R0, acc, ring, sum, comp);
            } else {
                belt_block<false>(sg, wbuf, j0, R0, acc, ring, sum, comp);
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    kahan(sum[u], comp[u], ring[u]);
                    ring[u] = 0.0f;
                }
            }
            j0 += 2 * kU;
        }
        for (; j0 < g.nd; j0 += 2 * kU) belt_block<false>(sg, wbuf, j0, R0, acc, ring, sum, comp);
#pragma unroll
        for (int u = 0; u < kU; ++u) kahan(sum[u], comp[u], ring[u]);
    }
    __syncthreads();
    if (*s_abort) {
        // wait (bounded) for any copy still in flight before leaving; a copy that
        // outlives that wait too is reported as such (it may still write the
        // buffers of a CTA that has exited)
        if (tid == 0) {
            const bool d0 = mbar_wait(&bar[0], phase0);
            const bool d1 = mbar_wait(&bar[1], phase1);
            atomicExch(err, d0 && d1 ? KSC_ERR_TIMEOUT : KSC_ERR_TIMEOUT_UNDRAINED);
        }
        return false;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const int k = k0 + kb + u;
        if (k < L) o[R.start + k] = sum[u] * P.domega;
    }
    return true;
}

// Shared state of a belt CTA: three seg_cap-float buffers (two input segments,
// the weight vector) in dynamic shared memory, two mbarriers.
#define KSC_BELT_SHARED_STATE                                           \
    extern __shared__ __align__(16) unsigned char smem_raw[];          \
    float *seg0 = reinterpret_cast<float *>(smem_raw);                  \
    float *seg1 = seg0 + seg_cap;                                       \
    float *wbuf = seg1 + seg_cap;                                       \
    __shared__ __align__(8) uint64_t bar[2];                            \
    __shared__ PairGeom s_g[2];                                         \
    __shared__ int s_abort;                                             \
    if (threadIdx.x == 0) {                                             \
        mbar_init(&bar[0], 1);                                          \
        mbar_init(&bar[1], 1);                                          \
        s_abort = 0;                                                    \
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); \
    }                                                                   \
    __syncthreads();                                                    \
    uint32_t phase0 = 0u, phase1 = 0u;

// One split, items assigned round-robin; grid.y runs over maps.
template <int T>
__global__ void __launch_bounds__(T)
conv_belt_kernel(const ConvPlan P, const int2 *__restrict__ items, int n_items,
                 const float *__restrict__ in, float *__restrict__ out, long long map_stride,
                 int seg_cap, int *__restrict__ err) {
    KSC_BELT_SHARED_STATE
    const float *m = in + (long long)blockIdx.y * map_stride;
    float *o = out + (long long)blockIdx.y * map_stride;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        if (!belt_item<T>(P, items[it].x, items[it].y, m, o, seg0, seg1, wbuf, bar, s_g,
                          &s_abort, phase0, phase1, seg_cap, err))
            return;
    }
}

// A batch of (split, map) entries: persistent CTAs claim items (entry, ring,
// first pixel) from a global counter, in the order of the list (longest
// first), until the list is exhausted.
template <int T>
__global__ void __launch_bounds__(T)
conv_belt_batch_kernel(const ConvPlan *__restrict__ plans, const BatchEntry *__restrict__ entries,
                       const int4 *__restrict__ items, int n_items, int seg_cap,
                       int *__restrict__ err, int *__restrict__ counter) {
    KSC_BELT_SHARED_STATE
    __shared__ int s_next;
    for (;;) {
        __syncthreads();  // every thread has read the previous claim
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_next;
        if (it >= n_items) break;
        const int4 w = items[it];
        const BatchEntry e = entries[w.x];
        if (!belt_item<T>(plans[e.plan], w.y, w.z, e.in, e.out, seg0, seg1, wbuf, bar, s_g,
                          &s_abort, phase0, phase1, seg_cap, err))
            return;
    }
}

#undef KSC_BELT_SHARED_STATE

int sm_count() {
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    return n_sm;
}

template <class K>
cudaError_t belt_grid(K kernel, int threads, size_t smem, int n_items, int per_sm_cap,
                      int *blocks) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
    if (per_sm < 1) per_sm = 1;
    *blocks = std::min(sm_count() * per_sm, n_items);
    return cudaSuccess;
}

} // namespace

int belt_chunk() { return kChunk; }

cudaError_t launch_conv_belt(const ConvPlan &p, const int2 *d_items, int n_items, int seg_cap,
                             const float *d_in, float *d_out, int n_maps, long long map_stride,
                             int *d_err, cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * 3 * (size_t)seg_cap;
    int blocks = 0;
    cudaError_t e = belt_grid(conv_belt_kernel<kThreads>, kThreads, smem, n_items, 0, &blocks);
    if (e != cudaSuccess) return e;
    dim3 grid(blocks, n_maps);
    conv_belt_kernel<kThreads><<<grid, kThreads, smem, st>>>(p, d_items, n_items, d_in, d_out,
                                                             map_stride, seg_cap, d_err);
    return cudaGetLastError();
}

int belt_variant_chunk(int variant) { return kU * (variant == 1 ? kThreads / 2 : kThreads); }

cudaError_t launch_conv_belt_batch(int variant, const ConvPlan *d_plans,
                                   const BatchEntry *d_entries, const int4 *d_items, int n_items,
                                   int seg_cap, int per_sm_cap, int *d_err, int *d_counter,
                                   cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * 3 * (size_t)seg_cap;
    int blocks = 0;
    cudaError_t e;
    if (variant == 1) {
        constexpr int T = kThreads / 2;
        e = belt_grid(conv_belt_batch_kernel<T>, T, smem, n_items, per_sm_cap, &blocks);
        if (e != cudaSuccess) return e;
        conv_belt_batch_kernel<T><<<blocks, T, smem, st>>>(d_plans, d_entries, d_items, n_items,
                                                           seg_cap, d_err, d_counter);
    } else {
        constexpr int T = kThreads;
        e = belt_grid(conv_belt_batch_kernel<T>, T, smem, n_items, per_sm_cap, &blocks);
        if (e != cudaSuccess) return e;
        conv_belt_batch_kernel<T><<<blocks, T, smem, st>>>(d_plans, d_entries, d_items, n_items,
                                                           seg_cap, d_err, d_counter);
    }
    return cudaGetLastError();
}

} // namespace ksc
