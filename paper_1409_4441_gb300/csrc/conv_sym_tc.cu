// Real-space convolution of the symmetric (cap) ring pairs for one map with the
// pixel-pair products on the tcgen05 tensor cores.
//
// Per input ring q, the 128 reflection classes k of an item of output ring r
// and the sixteen symmetry images n of input position k' (the same image
// permutations as the FFMA gather, conv_sym.cu) form a contraction
//
//   D[k][n] += sum_k' W[k][k'] X[n][k'],    W[k][k'] = K_r(chord(k, k')),
//
// over the positions k' of the classes' union window: M = 128 classes, N = 16
// images, K = 16 positions per MMA step.  W is evaluated by one thread per class
// row from the ring pair's table in |N| (ksc_sym.cuh) -- the same weights as the
// FFMA gather -- and written to tensor memory (tcgen05.st), where the MMA reads
// A; X is staged once per ring pair in shared memory in the canonical K-major
// layout, where the MMA reads B.  The tensor core thus does the multiply-adds
// and the image traffic, and the threads only look up weights.
//
// FP32 accuracy from BF16 operands: every weight and every image value is split
// exactly into three BF16 parts by truncation, w = w1 + w2 + w3 (8 + 8 + 8
// significand bits; w - w1 and its remainder are exact in FP32), and the
// product keeps the six terms of order up to 2^-16: w1 x1 in a fresh accumulator
// per step, w1 x2 + w2 x1 + w1 x3 + w2 x2 + w3 x1 (2^-8 of the first) in a second
// accumulator over the segment.  BF16 products are exact in the FP32
// accumulator, so each step's leading term carries one accumulator rounding of
// a 16-term sum; it is drained every step into FP32 partials, which are
// Kahan-folded into the totals every 64 positions as in the FFMA gather.
//
// Warps 0-3 own the 128 class rows (a warp reaches TMEM lanes 32 w .. 32 w + 31);
// warp 4 allocates tensor memory and one of its threads issues the MMAs.  Two
// A / D buffers let one step's MMAs run while the next step's weights are
// written.  Every mbarrier wait is bounded: a wait that runs out raises the
// device error flag and the CTA stops, drains (bounded) its MMAs and frees its
// tensor memory only if they completed.
#include <cstdint>

#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_sym.cuh"
#include "ksc_tc.cuh"

namespace ksc {
namespace {

constexpr int kM = 128;             // classes per item (TMEM lanes)
constexpr int kN = 16;              // symmetry images (accumulator columns)
constexpr int kK = 16;              // positions per MMA step (BF16 K)
constexpr int kRows = kM;           // threads that own class rows
constexpr int kThreads = kRows + 32;  // + the MMA warp
constexpr int kSpan = 448;          // staged positions per segment (multiple of kK)
constexpr int kKG = kSpan / 8;      // 8-position core-matrix groups per staged row group
constexpr int kRingChunk = 32;
constexpr int kFoldSteps = 4;       // steps per Kahan fold (64 positions)
constexpr int kNB = 4;              // A / D buffers (steps in flight)
// tensor memory columns: A[b][t] (t = split), D[b] (leading term), X (cross terms)
constexpr uint32_t kColA = 0, kColD = 24 * kNB, kColX = kColD + 16 * kNB, kTmemCols = 256;
static_assert(kColX + 16 <= kTmemCols, "tensor memory budget");
constexpr uint32_t kSplitBytes = 2u * kKG * 128u;  // one BF16 split of the staged images
static_assert(kSpan % kK == 0, "segments hold whole steps");

// instruction descriptor: F32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// B descriptor of the staged split starting at byte address `a` (core matrices
// of 8 images x 8 positions, K-adjacent ones 128 B apart, the second 8-image
// group kKG * 128 B further).
__device__ __forceinline__ uint64_t bdesc(uint32_t a) {
    uint64_t d = 0;
    d |= (uint64_t)((a & 0x3FFFF) >> 4);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)(((kKG * 128u) >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t db,
                                            uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::saddr(bar)) : "memory");
}

// Exact three-way BF16 split of two FP32 values, packed per split: word t holds
// part t of a in its low half and part t of b in its high half.
__device__ __forceinline__ void split3_pack(float a, float b, uint32_t *p1, uint32_t *p2,
                                            uint32_t *p3) {
    const uint32_t m = 0xFFFF0000u;
    const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
    *p1 = __byte_perm(ua, ub, 0x7632);
    const float ra = a - __uint_as_float(ua & m), rb = b - __uint_as_float(ub & m);
    const uint32_t va = __float_as_uint(ra), vb = __float_as_uint(rb);
    *p2 = __byte_perm(va, vb, 0x7632);
    const float sa = ra - __uint_as_float(va & m), sb = rb - __uint_as_float(vb & m);
    *p3 = __byte_perm(__float_as_uint(sa), __float_as_uint(sb), 0x7632);
}

__device__ __forceinline__ void kahan(float *sum, float *comp, float v) {
    const float y = v - *comp;
    const float tt = *sum + y;
    *comp = (tt - *sum) - y;
    *sum = tt;
}

__device__ __forceinline__ int floor_div(int a, int b) {
    const int q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}
__device__ __forceinline__ int ceil_div(int a, int b) {
    const int q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}

// The sixteen weights of positions p0 .. p0 + 15 for one class.  Table path: the
// ring pair's table with its last cell ending at the cut (xtab_build_cut), looked
// up at min(|N| + off, nct 2^shift) in table units (offS = off 2^-shift, ncf =
// nct): K_r within the cut, exactly 0 beyond, the same branch-free code for every
// position.  Per-pair path: the double-float chord, zero outside [wa, wb] and
// beyond the cut.  Returns false when every lane of the warp has only zero weights
// (its window misses the step; the caller then writes zeros).
__device__ __forceinline__ bool step_weights(const ConvPlan &P, const SymRing &g,
                                             const float4 *xt, bool use_xt, float offS,
                                             float ncf, int p0, int wa, int wb, int num, int L,
                                             float *w) {
    if (__all_sync(~0u, p0 > wb || p0 + kK - 1 < wa)) return false;
    if (use_xt) {
        // exact wherever |N| + off stays below the cut cell: |N| < 2^24 near the window
        const float step = (float)(2 * L) * g.inv;
        const float tp = (float)(num - 2 * L * p0) * g.inv;
#pragma unroll
        for (int e = 0; e < kK; ++e)
            w[e] = xtab_at(xt, fminf(fabsf(fmaf(-(float)e, step, tp)) + offS, ncf));
    } else {
        const float N0 = (float)(num - 2 * L * p0);
        const float stepf = (float)(2 * L);
        if (g.small) {
#pragma unroll
            for (int e = 0; e < kK; ++e)
                w[e] = sym_weight<true>(P, g, N0 - (float)e * stepf, p0 + e, wa, wb);
        } else {
#pragma unroll
            for (int e = 0; e < kK; ++e)
                w[e] = sym_weight<false>(P, g, N0 - (float)e * stepf, p0 + e, wa, wb);
        }
    }
    return true;
}

// Stage the sixteen image sequences of positions s0 .. s0 + span - 1 of input ring g
// as three BF16 splits in the canonical K-major layout: image n, position j at
// split + ((n >> 3) kKG + (j >> 3)) * 128 + (n & 7) * 16 + (j & 7) * 2 bytes.
// Images: 0-3 direct quarter turns, 4-7 their mirror ring, 8-11 reflected, 12-15
// reflected on the mirror ring (zero on the equator, which has no mirror).
__device__ __forceinline__ void stage_images(const float *__restrict__ m, const SymRing &g,
                                             bool mirror, int s0, int span, unsigned char *bs) {
    const int L2 = g.len, Q2 = L2 / 4;
    const int n_tasks = kN * (span / 8);
    for (int task = threadIdx.x; task < n_tasks; task += kThreads) {
        const int n = task & (kN - 1), c = task >> 4;
        const int qq = n & 3;
        const bool south = (n >> 2) & 1, refl = n >> 3;
        float v[8];
        if (south && !mirror) {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = 0.0f;
        } else {
            const float *ring = m + (south ? g.start_m : g.start);
            const int kp = s0 + 8 * c;
            const int base = (refl ? Q2 - kp - g.phase : kp) + qq * Q2;
            if (L2 >= 8) {  // one wrap per index at most
                const int b0 = sym_pmod(base, L2);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    int ix = refl ? b0 - e : b0 + e;
                    ix += ix < 0 ? L2 : 0;
                    ix -= ix >= L2 ? L2 : 0;
                    v[e] = __ldg(ring + ix);
                }
            } else {  // rings of 4 pixels at the poles: reduce every index
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[e] = __ldg(ring + sym_pmod(refl ? base - e : base + e, L2));
            }
        }
        uint32_t p1[4], p2[4], p3[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split3_pack(v[2 * j], v[2 * j + 1], &p1[j], &p2[j], &p3[j]);
        const uint32_t off = (uint32_t)(((n >> 3) * kKG + c) * 128 + (n & 7) * 16);
        *reinterpret_cast<uint4 *>(bs + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
        *reinterpret_cast<uint4 *>(bs + kSplitBytes + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
        *reinterpret_cast<uint4 *>(bs + 2 * kSplitBytes + off) =
            make_uint4(p3[0], p3[1], p3[2], p3[3]);
    }
}

__global__ void __launch_bounds__(kThreads, 2)
conv_sym_tc_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                   const float *__restrict__ in, float *__restrict__ out, long long map_stride,
                   int belt_split, int band_lo, int band_hi, int *__restrict__ counters,
                   int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *bs = smem_raw;  // 3 BF16 splits of the staged images
    float4 *xt = reinterpret_cast<float4 *>(smem_raw + 3 * kSplitBytes);  // kXCap cells
    __shared__ SymRing sR[kRingChunk];
    __shared__ __align__(8) uint64_t a_full[kNB], mma_done[kNB];
    __shared__ uint32_t tmem_base;
    __shared__ int s_next, s_abort, s_drained;

    const int tid = threadIdx.x, warp = tid >> 5;
    const bool row_thread = tid < kRows;
    const bool issuer = tid == kRows;
    const float *m = in + (long long)blockIdx.y * map_stride;
    float *o = out + (long long)blockIdx.y * map_stride;
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::saddr(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < kNB; ++b) {
            tc::mbar_init(&a_full[b], kRows);
            tc::mbar_init(&mma_done[b], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_drained = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t idesc = idesc_bf16(kM, kN);
    const uint32_t bs_addr = tc::saddr(bs);
    // per-buffer state as bit masks (bit b: buffer b): mbarrier phases, and for the
    // row threads the buffers whose MMAs are not yet drained
    uint32_t ph_done = 0u, ph_full = 0u, pending = 0u;
    // row warps: buffers whose A rows of this warp hold zeros (no store needed), and
    // steps in flight whose rows were all zero (D rows zero: no drain needed)
    uint32_t a_zero = 0u, d_zero = 0u;
    bool ok = true;
    const int eq = (P.nrings - 1) / 2;

    for (;;) {
        __syncthreads();  // every thread has read the previous claim
        if (tid == 0) s_next = atomicAdd(&counters[blockIdx.y], 1);
        __syncthreads();
        const int it = s_next;
        if (it >= n_items || s_abort) break;
        const WorkItem wi = items[it];
        const int r = wi.ring, c0 = wi.k0;
        const DevRing R = P.d_rings[r];
        const int L = R.len, Q = L / 4, t = R.phase;
        const int2 rg = P.d_range[r];
        const int n_cls = t ? (Q + 1) / 2 : Q / 2 + 1;
        const bool mirror = r != eq;
        const bool add = belt_split && r >= P.belt_lo && r <= P.belt_hi;
        const int k = c0 + (tid & (kRows - 1));
        const bool active = row_thread && k < n_cls;
        const int k_first = c0, k_last = min(c0 + kM, n_cls) - 1;
        const int kb = Q - k - t;
        const bool refl = kb != k && kb != Q;
        float sum[kN], comp[kN], part[kN];
#pragma unroll
        for (int i = 0; i < kN; ++i) sum[i] = comp[i] = part[i] = 0.0f;
        int nfold = 0;

        for (int q0 = rg.x; q0 <= rg.y && ok; q0 += kRingChunk) {
            const int nq = min(kRingChunk, rg.y - q0 + 1);
            __syncthreads();
            if (tid < nq) sR[tid] = load_sym_ring(P, r, q0 + tid, rg, add);
            __syncthreads();
            for (int qi = 0; qi < nq && ok; ++qi) {
                const SymRing g = sR[qi];
                if (g.hw < 0.0f) continue;
                long long numl, numx;
                int klo, khi, U0, U1, dummy;
                sym_window(k, t, L, g, &numl, &klo, &khi);
                sym_window(k_first, t, L, g, &numx, &U0, &dummy);
                sym_window(k_last, t, L, g, &numx, &dummy, &U1);
                const int num = (int)numl;  // < 2^31 for nside <= 8192
                // table with its last cell ending at the cut (plus one zero cell)
                const int off = (-(g.ncut + 1)) & ((1 << g.shift) - 1);
                const int nct = (g.ncut + 1 + off) >> g.shift;
                const bool use_xt = g.ncell > 0 && nct + 1 <= kXCap;
                const float offS = (float)off * g.inv, ncf = (float)nct;
                // invariants the arithmetic relies on (guaranteed by the split's
                // construction): class integers fit in int32, and table positions within
                // a step of the cut stay exact in FP32
                if (tid == 0 && (numx + 2LL * kM * g.len > 2147483647LL ||
                                 (use_xt && (long long)g.ncut + 32LL * L >= (1LL << 24))))
                    atomicExch(err, KSC_ERR_DEVICE_BOUNDS);
                int wa = klo, wb = khi;
                if (use_xt) {  // the class's positions within the cut
                    wa = max(klo, ceil_div(num - g.ncut, 2 * L));
                    wb = min(khi, floor_div(num + g.ncut, 2 * L));
                }
                if (!active) {  // no weights: zero rows
                    wa = 1;
                    wb = 0;
                }
                if (use_xt) {
                    __syncthreads();  // the previous ring pair's lookups are done
                    xtab_build_cut<kThreads>(P, g, xt, off, nct);
                }
                for (int s0 = U0 & ~(kK - 1); s0 <= U1 && ok; s0 += kSpan) {
                    const int span = min(kSpan, ((U1 - s0 + 1) + kK - 1) & ~(kK - 1));
                    const int n_steps = span / kK;
                    __syncthreads();  // the previous segment's MMAs have completed
                    stage_images(m, g, mirror, s0, span, bs);
                    tc::fence_async_smem();
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    bool bad = false;  // a bounded wait of this warp ran out
                    if (row_thread) {
                        for (int s = 0; s < n_steps; ++s) {
                            const int b = s % kNB;
                            if ((pending >> b) & 1u) {  // drain this buffer's previous step
                                if (!__all_sync(~0u, tc::mbar_wait(&mma_done[b],
                                                                   (ph_done >> b) & 1u))) {
                                    s_abort = 1;
                                    bad = true;
                                    break;
                                }
                                ph_done ^= 1u << b;
                                pending &= ~(1u << b);
                                tc::fence_after_sync();
                                if (!((d_zero >> b) & 1u)) {
                                    uint32_t d[kN];
                                    tc::tmem_ld16(tmem + lane + kColD + 16u * b, d);
                                    tc::tmem_wait_ld();
#pragma unroll
                                    for (int i = 0; i < kN; ++i) part[i] += __uint_as_float(d[i]);
                                }
                                if (++nfold == kFoldSteps) {
                                    nfold = 0;
#pragma unroll
                                    for (int i = 0; i < kN; ++i) {
                                        kahan(&sum[i], &comp[i], part[i]);
                                        part[i] = 0.0f;
                                    }
                                }
                            }
                            float w[kK];
                            const uint32_t ta = tmem + lane + kColA + 24u * b;
                            if (step_weights(P, g, xt, use_xt, offS, ncf, s0 + kK * s, wa, wb,
                                             num, L, w)) {
                                uint32_t a1[8], a2[8], a3[8];
#pragma unroll
                                for (int j = 0; j < 8; ++j)
                                    split3_pack(w[2 * j], w[2 * j + 1], &a1[j], &a2[j], &a3[j]);
                                __syncwarp();
                                tmem_st8(ta, a1);
                                tmem_st8(ta + 8u, a2);
                                tmem_st8(ta + 16u, a3);
                                tc::tmem_wait_st();
                                a_zero &= ~(1u << b);
                                d_zero &= ~(1u << b);
                            } else {  // every row of this warp is zero in this step
                                if (!((a_zero >> b) & 1u)) {
                                    uint32_t z[8];
#pragma unroll
                                    for (int j = 0; j < 8; ++j) z[j] = 0u;
                                    __syncwarp();
                                    tmem_st8(ta, z);
                                    tmem_st8(ta + 8u, z);
                                    tmem_st8(ta + 16u, z);
                                    tc::tmem_wait_st();
                                    a_zero |= 1u << b;
                                }
                                d_zero |= 1u << b;
                            }
                            tc::fence_before_sync();
                            mbar_arrive(&a_full[b]);
                            pending |= 1u << b;
                        }
                        // drain the last steps: the leading terms, then the cross terms
                        for (int bb = 0; bb < kNB && !bad; ++bb) {
                            const int b = (n_steps + bb) % kNB;  // older buffers first
                            if (!((pending >> b) & 1u)) continue;
                            if (!__all_sync(~0u, tc::mbar_wait(&mma_done[b],
                                                               (ph_done >> b) & 1u))) {
                                s_abort = 1;
                                bad = true;
                                break;
                            }
                            ph_done ^= 1u << b;
                            pending &= ~(1u << b);
                            tc::fence_after_sync();
                            if (!((d_zero >> b) & 1u)) {
                                uint32_t d[kN];
                                tc::tmem_ld16(tmem + lane + kColD + 16u * b, d);
                                tc::tmem_wait_ld();
#pragma unroll
                                for (int i = 0; i < kN; ++i) part[i] += __uint_as_float(d[i]);
                            }
                        }
                        if (!bad) {
                            uint32_t x[kN];
                            tc::tmem_ld16(tmem + lane + kColX, x);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int i = 0; i < kN; ++i) {
                                part[i] += __uint_as_float(x[i]);
                                kahan(&sum[i], &comp[i], part[i]);
                                part[i] = 0.0f;
                            }
                            nfold = 0;
                        }
                    } else if (issuer) {
                        for (int s = 0; s < n_steps; ++s) {
                            const int b = s % kNB;
                            if (!tc::mbar_wait_sleep(&a_full[b], (ph_full >> b) & 1u, 1000u)) {
                                s_abort = 1;
                                break;
                            }
                            ph_full ^= 1u << b;
                            tc::fence_after_sync();
                            const uint32_t ta = tmem + kColA + 24u * b;
                            const uint32_t td = tmem + kColD + 16u * b, tx = tmem + kColX;
                            const uint32_t kb_off = (uint32_t)(s * (kK / 8) * 128);
                            const uint64_t b1 = bdesc(bs_addr + kb_off);
                            const uint64_t b2 = bdesc(bs_addr + kSplitBytes + kb_off);
                            const uint64_t b3 = bdesc(bs_addr + 2 * kSplitBytes + kb_off);
                            mma_bf16_ts(td, ta, b1, idesc, 0u);              // w1 x1 (fresh)
                            mma_bf16_ts(tx, ta, b2, idesc, s > 0 ? 1u : 0u);  // w1 x2
                            mma_bf16_ts(tx, ta + 8u, b1, idesc, 1u);        // w2 x1
                            mma_bf16_ts(tx, ta, b3, idesc, 1u);             // w1 x3
                            mma_bf16_ts(tx, ta + 8u, b2, idesc, 1u);        // w2 x2
                            mma_bf16_ts(tx, ta + 16u, b1, idesc, 1u);       // w3 x1
                            tc::mma_commit(&mma_done[b]);
                        }
                    }
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    if (s_abort) ok = false;
                }
            }
        }
        if (!ok) break;
        if (active) {
            const int rs = P.nrings - 1 - r;
            const int start_s = P.d_rings[rs].start;
            const bool wn = r >= band_lo && r <= band_hi;
            const bool ws = mirror && rs >= band_lo && rs <= band_hi;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (c == 1 && !refl) break;
                const int kk = c ? kb : k;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const int kq = kk + qq * Q;
                    const float vn = sum[8 * c + qq] * P.domega;
                    if (wn) {
                        if (add) o[R.start + kq] += vn;
                        else o[R.start + kq] = vn;
                    }
                    if (mirror) {
                        const float vs = sum[8 * c + 4 + qq] * P.domega;
                        if (ws) {
                            if (add) o[start_s + kq] += vs;
                            else o[start_s + kq] = vs;
                        }
                    }
                }
            }
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, KSC_ERR_TIMEOUT);
        // bounded drain of MMAs still in flight (a commit tracks every earlier MMA of
        // its thread); tensor memory that one of them may still write is not freed
        if (row_thread)
            for (int b = 0; b < kNB; ++b)
                if (((pending >> b) & 1u) && !tc::mbar_wait(&mma_done[b], (ph_done >> b) & 1u))
                    s_drained = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && !s_drained) atomicExch(err, KSC_ERR_TIMEOUT_UNDRAINED);
    if (warp == 4 && s_drained)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

} // namespace

int sym_tc_chunk() { return kM; }

cudaError_t launch_conv_sym_tc(const ConvPlan &p, const WorkItem *d_items, int n_items,
                               const float *d_in, float *d_out, int n_maps, long long map_stride,
                               int belt_split, int band_lo, int band_hi, int *d_err,
                               cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    const size_t smem = 3 * (size_t)kSplitBytes + sizeof(float4) * kXCap;
    cudaError_t e = cudaFuncSetAttribute(conv_sym_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // two CTAs per SM: shared memory (table + staged images) and tensor memory
    // (256 of 512 columns) are sized for that; CTAs claim items, so a CTA that
    // cannot be resident yet only starts later
    const int blocks = n_items < 2 * n_sm ? n_items : 2 * n_sm;
    int *ctr = nullptr;
    const size_t bytes = sizeof(int) * (size_t)n_maps;
    if ((e = cudaMallocAsync(&ctr, bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ctr, 0, bytes, st)) == cudaSuccess) {
        dim3 grid(blocks, n_maps);
        conv_sym_tc_kernel<<<grid, kThreads, smem, st>>>(p, d_items, n_items, d_in, d_out,
                                                         map_stride, belt_split, band_lo, band_hi,
                                                         ctr, d_err);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(ctr, st);
    return e != cudaSuccess ? e : f;
}

} // namespace ksc
