// Map stacks: the symmetric (cap) ring pairs on the tcgen05 tensor cores.
//
// The FFMA gather (conv_sym.cu) evaluates each kernel weight w(k, k') once per
// map and uses it for the sixteen symmetry images of that map.  For a stack of
// maps sharing one split the weight depends on neither the image nor the map,
// so the contribution of input ring q to 128 reflection classes of output ring
// r is a dense contraction
//
//   D[k][n] += sum_k' W[k][k'] X[n][k'],   n = (image, map),
//
// over the positions k' of the classes' union window: A = W (128 classes x 32
// positions per K tile, zero outside each class's window and beyond the cut),
// B = X (16 images x 8 maps = 128 rows x 32 positions, gathered with the
// image permutations: quarter turns, mirror ring, reflection).  M = N = 128,
// TF32 x3 (hi*hi + hi*lo + lo*hi, FP32 products to about 2^-22) with FP32
// accumulation in tensor memory; after each ring pair the partial accumulator
// is Kahan-folded into running sums kept in tensor memory too (columns
// [0, 128) partial, [128, 256) sum, [256, 384) compensation).  Four threads per
// class row build the operand tiles (the weight evaluation is the cost), the
// operand stages are double-buffered so one tile's MMAs overlap the next
// tile's build, and every mbarrier wait is bounded: on a timeout the kernel
// raises the device error flag, drains its MMAs and frees its tensor memory.
#include <cstdint>

#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_sym.cuh"
#include "ksc_tc.cuh"

namespace ksc {
namespace {

constexpr int kM = 128;           // classes per item (TMEM lanes)
constexpr int kImg = 16;          // symmetry images
constexpr int kMaps = 8;          // maps per group
constexpr int kN = kImg * kMaps;  // accumulator columns, n = image * kMaps + map
constexpr int kKT = 32;           // positions per K tile (4 MMAs of K = 8)
constexpr int kThreads = 512;     // four threads per class row
constexpr int kParts = kThreads / kM;
constexpr int kRingChunk = 32;
constexpr uint32_t kColSum = kN, kColCmp = 2 * kN, kTmemCols = 512;

struct Stage {  // canonical no-swizzle K-major tiles
    float a_hi[kM * kKT], a_lo[kM * kKT];
    float b_hi[kN * kKT], b_lo[kN * kKT];
};

__device__ __forceinline__ void store_split4(float *hi, float *lo, int off, float4 v) {
    float h[4], l[4];
    tc::split_tf32(v.x, &h[0], &l[0]);
    tc::split_tf32(v.y, &h[1], &l[1]);
    tc::split_tf32(v.z, &h[2], &l[2]);
    tc::split_tf32(v.w, &h[3], &l[3]);
    *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
}

// A tile row `row`, quads part, part + 4 of the tile (positions pbase + 4 qd ..
// + 3): weights of class k (integer num, window [a, b]).  The four threads of
// a row interleave quads so all see the same share of the class's window;
// quads wholly outside the window are zero without evaluation (the tiles span
// the union of 128 classes' windows, whose ends shift by about one position
// per class, so the branch is uniform across a warp except near the ends).
// MODE 0 / 1: double-float chord (general / small-angle sine); 2: the ring
// pair's x table xt (partial windows: positions outside [a, b] lie beyond the
// cut, which the table's cut test zeroes).
template <int MODE>
__device__ __forceinline__ void build_a(const ConvPlan &P, const SymRing &g, const float4 *xt,
                                        Stage &S, int row, int part, int pbase, long long num,
                                        int L, int a, int b) {
    const float step = (float)(2 * L);
#pragma unroll
    for (int j = 0; j < (kKT / 4) / kParts; ++j) {
        const int qd = part + kParts * j;
        const int kq = pbase + 4 * qd;
        const int o = tc::toff<kKT>(row, 4 * qd);
        if (kq + 3 < a || kq > b) {
            *reinterpret_cast<float4 *>(S.a_hi + o) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            *reinterpret_cast<float4 *>(S.a_lo + o) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            continue;
        }
        const float N0 = (float)(num - 2LL * kq * L);
        float4 w;
        if constexpr (MODE == 2) {
            w.x = xtab_weight(xt, g, N0);
            w.y = xtab_weight(xt, g, N0 - step);
            w.z = xtab_weight(xt, g, N0 - 2.0f * step);
            w.w = xtab_weight(xt, g, N0 - 3.0f * step);
        } else {
            w.x = sym_weight<MODE == 1>(P, g, N0, kq, a, b);
            w.y = sym_weight<MODE == 1>(P, g, N0 - step, kq + 1, a, b);
            w.z = sym_weight<MODE == 1>(P, g, N0 - 2.0f * step, kq + 2, a, b);
            w.w = sym_weight<MODE == 1>(P, g, N0 - 3.0f * step, kq + 3, a, b);
        }
        store_split4(S.a_hi, S.a_lo, o, w);
    }
}

// This lane's 8 B-tile values (two rows, four positions) of the tile starting
// at pbase (see the assignment in the kernel).
__device__ __forceinline__ void load_b(const float *const *src, int qoff, const bool *live,
                                       bool reflected, int pbase, int pg, int L2, int Q2, int phase,
                                       float *v) {
    const int pp = pbase + 4 * pg;
    const int base = reflected ? sym_pmod(Q2 - pp - phase, L2) : sym_pmod(pp, L2);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        int ix = reflected ? base - e : base + e;
        ix += ix < 0 ? L2 : 0;
        ix -= ix >= L2 ? L2 : 0;
        ix += qoff;
        ix -= ix >= L2 ? L2 : 0;
#pragma unroll
        for (int i = 0; i < 2; ++i) v[4 * i + e] = live[i] ? __ldg(src[i] + ix) : 0.0f;
    }
}

__global__ void __launch_bounds__(kThreads, 1)
conv_sym_mma_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                    const float *__restrict__ in, float *__restrict__ out, int n_maps,
                    long long map_stride, int belt_split, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Stage *stage = reinterpret_cast<Stage *>(smem_raw);  // 2 stages
    float4 *xt = reinterpret_cast<float4 *>(smem_raw + 2 * sizeof(Stage));  // kXCap cells
    __shared__ SymRing sR[kRingChunk];
    __shared__ __align__(8) uint64_t mdone[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ int s_drained;  // 0: an MMA outlived the bounded drain

    const int tid = threadIdx.x, warp = tid >> 5;
    // Epilogue (tensor memory) mapping: a warp reaches TMEM lanes 32 (warp % 4) ..
    // + 31, so warp w holds class rows 32 (w % 4) .. and column part w / 4.
    const int row = tid & (kM - 1), part = tid >> 7;
    // A-tile mapping: warp w builds rows 32 (w / 4) .. + 31, quads part w % 4, so
    // each scheduler (warps w = s mod 4) holds every row block and the rows whose
    // windows miss a tile (at the ends of the union) spread over all schedulers.
    const int brow = (tid & 31) + 32 * (warp >> 2), bpart = warp & 3;
    const int grp = blockIdx.y;                        // map group
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc::saddr(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        tc::mbar_init(&mdone[0], 1);
        tc::mbar_init(&mdone[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_drained = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;  // this warp's TMEM lanes
    const uint32_t idesc = tc::idesc_tf32(kM, kN);
    uint32_t ph_done[2] = {0u, 0u};
    int pending[2] = {0, 0};
    int tcount = 0;
    bool ok = true;
    const int eq = (P.nrings - 1) / 2;  // the equator ring, its own mirror image
    const uint32_t zero16[16] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};

    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        const WorkItem wi = items[it];
        const int r = wi.ring, c0 = wi.k0;
        const DevRing R = P.d_rings[r];
        const int L = R.len, Q = L / 4, t = R.phase;
        const int2 rg = P.d_range[r];
        const int n_cls = t ? (Q + 1) / 2 : Q / 2 + 1;
        const bool mirror = r != eq;
        const bool add = belt_split && r >= P.belt_lo && r <= P.belt_hi;
        const int k = c0 + row;
        const bool active = k < n_cls;
        const int kbld = c0 + brow;  // class of the A-tile row this thread builds
        const int k_first = c0, k_last = min(c0 + kM, n_cls) - 1;
        const int kb = Q - k - t;
        const bool refl = kb != k && kb != Q;
        // running sums and compensations of this warp's lanes, its column part
#pragma unroll
        for (int cc = 0; cc < kN / kParts; cc += 16) {
            const uint32_t col = (uint32_t)(part * (kN / kParts) + cc);
            tc::tmem_st16(tmem + lane + kColSum + col, zero16);
            tc::tmem_st16(tmem + lane + kColCmp + col, zero16);
        }
        tc::tmem_wait_st();

        for (int q0 = rg.x; q0 <= rg.y && ok; q0 += kRingChunk) {
            const int nq = min(kRingChunk, rg.y - q0 + 1);
            tc::fence_before_sync();
            __syncthreads();
            if (tid < nq) sR[tid] = load_sym_ring(P, r, q0 + tid, rg, add);
            __syncthreads();
            tc::fence_after_sync();
            for (int qi = 0; qi < nq && ok; ++qi) {
                const SymRing g = sR[qi];
                if (g.hw < 0.0f) continue;
                const int L2 = g.len, Q2 = L2 / 4;
                long long num, numx;
                int klo, khi, U0, U1, dummy;
                sym_window(kbld, t, L, g, &num, &klo, &khi);
                sym_window(k_first, t, L, g, &numx, &U0, &dummy);
                sym_window(k_last, t, L, g, &numx, &dummy, &U1);
                if (kbld >= n_cls) {  // empty window: zero weights
                    klo = 1;
                    khi = 0;
                }
                const bool use_xt = g.ncell > 0 && g.ncell <= kXCap;
                // invariants the arithmetic relies on (guaranteed by the split's
                // construction): pixel-pair integers near the window exact in FP32
                if (tid == 0 && (numx + 2LL * kM * g.len > 2147483647LL ||
                                 (use_xt && (long long)g.ncut + 32LL * L >= (1LL << 24))))
                    atomicExch(err, KSC_ERR_DEVICE_BOUNDS);
                if (use_xt) {  // (the previous ring pair ended at a barrier)
                    xtab_build<kThreads>(P, g, xt);
                    __syncthreads();
                }
                const int P0 = U0 & ~(kKT - 1);
                const int n_tiles = (U1 - P0) / kKT + 1;
                // B tile assignment: warp w gathers image w (direct for w < 8,
                // reflected after; north for w % 8 < 4) for the 8 maps: lane l takes
                // positions 4 (l % 8) .. +3 of rows n = 8 w + l / 8 + 4 i, i = 0, 1
                // (n = image * kMaps + map): 8 lanes cover a row's 32 positions.
                const int lane_id = tid & 31;
                const int pg = lane_id & 7, sub = lane_id >> 3;
                const bool reflected = warp >= 8;
                const bool south = (warp >> 2) & 1;
                const bool b_live_hemi = mirror || !south;
                const int qoff = (warp & 3) * Q2;
                const float *src_base[2];
                bool live[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int mp = grp * kMaps + sub + 4 * i;
                    live[i] = b_live_hemi && mp < n_maps;
                    src_base[i] = live[i] ? in + (long long)mp * map_stride +
                                                (south ? g.start_m : g.start)
                                          : in;
                }
                float bv[8];  // this lane's B values of the current tile (prefetched)
                load_b(src_base, qoff, live, reflected, P0, pg, L2, Q2, g.phase, bv);
                for (int u = 0; u < n_tiles; ++u) {
                    const int b = tcount & 1;
                    bool stage_free = true;
                    if (pending[b]) {  // the MMAs that last read this stage are done
                        if (tc::mbar_wait(&mdone[b], ph_done[b])) {
                            ph_done[b] ^= 1u;
                            pending[b] = 0;
                        } else {  // still pending: write nothing into the stage
                            s_abort = 1;
                            stage_free = false;
                        }
                    }
                    Stage &S = stage[b];
                    const int pbase = P0 + u * kKT;
                    float bn[8];  // next tile's B values: loads in flight during the A build
                    if (u + 1 < n_tiles)
                        load_b(src_base, qoff, live, reflected, pbase + kKT, pg, L2, Q2, g.phase,
                               bn);
                    if (!stage_free) {
                    } else if (use_xt) {
                        build_a<2>(P, g, xt, S, brow, bpart, pbase, num, L, klo, khi);
                    } else if (g.small) {
                        build_a<1>(P, g, xt, S, brow, bpart, pbase, num, L, klo, khi);
                    } else {
                        build_a<0>(P, g, xt, S, brow, bpart, pbase, num, L, klo, khi);
                    }
                    if (stage_free) {
#pragma unroll
                        for (int i = 0; i < 2; ++i)
                            store_split4(S.b_hi, S.b_lo,
                                         tc::toff<kKT>(8 * warp + sub + 4 * i, 4 * pg),
                                         make_float4(bv[4 * i], bv[4 * i + 1], bv[4 * i + 2],
                                                     bv[4 * i + 3]));
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) bv[j] = bn[j];
                    tc::fence_async_smem();
                    tc::fence_before_sync();
                    __syncthreads();
                    tc::fence_after_sync();
                    if (s_abort) {  // uniform: read after the barrier
                        ok = false;
                        break;
                    }
                    if (tid == 0) {
#pragma unroll
                        for (int s = 0; s < kKT / 8; ++s) {
                            const uint64_t ah = tc::smem_desc<kKT>(S.a_hi + s * 64);
                            const uint64_t al = tc::smem_desc<kKT>(S.a_lo + s * 64);
                            const uint64_t bh = tc::smem_desc<kKT>(S.b_hi + s * 64);
                            const uint64_t bl = tc::smem_desc<kKT>(S.b_lo + s * 64);
                            const uint32_t acc = (u == 0 && s == 0) ? 0u : 1u;
                            tc::mma_tf32(tmem, ah, bh, idesc, acc);
                            tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                            tc::mma_tf32(tmem, al, bh, idesc, 1u);
                        }
                        tc::mma_commit(&mdone[b]);
                    }
                    pending[b] = 1;
                    ++tcount;
                }
                if (!ok) break;
                // every MMA of this ring pair has completed
                for (int bb = 0; bb < 2; ++bb) {
                    const int b = (tcount + bb) & 1;  // older stage first
                    if (pending[b]) {
                        if (tc::mbar_wait(&mdone[b], ph_done[b])) {
                            ph_done[b] ^= 1u;
                            pending[b] = 0;
                        } else {
                            s_abort = 1;
                        }
                    }
                }
                __syncthreads();
                if (s_abort) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                // Kahan-fold the partial into the running sums (this warp's lanes,
                // its column part)
#pragma unroll
                for (int cc = 0; cc < kN / kParts; cc += 16) {
                    const uint32_t col = (uint32_t)(part * (kN / kParts) + cc);
                    uint32_t pv[16], sv[16], cv[16];
                    tc::tmem_ld16(tmem + lane + col, pv);
                    tc::tmem_ld16(tmem + lane + kColSum + col, sv);
                    tc::tmem_ld16(tmem + lane + kColCmp + col, cv);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float s0 = __uint_as_float(sv[j]);
                        const float y = __uint_as_float(pv[j]) - __uint_as_float(cv[j]);
                        const float tt = s0 + y;
                        cv[j] = __float_as_uint((tt - s0) - y);
                        sv[j] = __float_as_uint(tt);
                    }
                    tc::tmem_st16(tmem + lane + kColSum + col, sv);
                    tc::tmem_st16(tmem + lane + kColCmp + col, cv);
                }
                tc::tmem_wait_st();
                tc::fence_before_sync();
            }
        }
        if (!ok) break;
        // outputs of class k: columns n = image * kMaps + map of this thread's part
        tc::fence_after_sync();
        const int rs = P.nrings - 1 - r;
        const int start_s = P.d_rings[rs].start;
#pragma unroll
        for (int cc = 0; cc < kN / kParts; cc += 16) {
            uint32_t sv[16];
            tc::tmem_ld16(tmem + lane + kColSum + (uint32_t)(part * (kN / kParts) + cc), sv);
            tc::tmem_wait_ld();
            if (!active) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = part * (kN / kParts) + cc + j;
                const int im = n / kMaps, mp = grp * kMaps + n % kMaps;
                const bool s_img = (im >> 2) & 1, r_img = im >> 3;
                if (mp >= n_maps || (r_img && !refl) || (s_img && !mirror)) continue;
                const int kk = (r_img ? kb : k) + (im & 3) * Q;
                float *o = out + (long long)mp * map_stride + (s_img ? start_s : R.start) + kk;
                const float v = __uint_as_float(sv[j]) * P.domega;
                if (add) *o += v;
                else *o = v;
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, KSC_ERR_TIMEOUT);
        // bounded drain of MMAs still in flight; if one never completes, the tensor
        // memory it may still write is not freed (see s_drained)
        for (int b = 0; b < 2; ++b)
            if (pending[b] && !tc::mbar_wait(&mdone[b], ph_done[b])) s_drained = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && !s_drained) atomicExch(err, KSC_ERR_TIMEOUT_UNDRAINED);
    if (warp == 0 && s_drained)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
}

} // namespace

int sym_mma_maps() { return kMaps; }

int sym_mma_chunk() { return kM; }

cudaError_t launch_conv_sym_mma(const ConvPlan &p, const WorkItem *d_items, int n_items,
                                const float *d_in, float *d_out, int n_maps,
                                long long map_stride, int belt_split, int *d_err,
                                cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    const size_t smem = 2 * sizeof(Stage) + sizeof(float4) * kXCap;
    cudaError_t e = cudaFuncSetAttribute(conv_sym_mma_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = n_sm;  // one CTA per SM (all 512 TMEM columns)
    if (blocks > n_items) blocks = n_items;
    dim3 grid(blocks, (n_maps + kMaps - 1) / kMaps);
    conv_sym_mma_kernel<<<grid, kThreads, smem, st>>>(p, d_items, n_items, d_in, d_out, n_maps,
                                                      map_stride, belt_split, d_err);
    return cudaGetLastError();
}

} // namespace ksc
