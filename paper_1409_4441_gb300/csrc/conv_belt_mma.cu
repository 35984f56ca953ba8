// Multi-map real-space convolution of belt ring pairs on the tcgen05 tensor
// cores (5th-generation MMA, accumulators in tensor memory).
//
// For n maps sharing one kernel, the contribution of belt input ring r' to a
// block of 128 consecutive outputs of belt ring r is a dense contraction
//
//   D[k][n] += sum_j W[k][j] X[n][j],   W[k][j] = w_{r r'}[p_j - k]
//
// over input positions p_j of ring r': the circulant kernel block (a Toeplitz
// band of the ring pair's weight vector, zero outside it) times the stack of
// maps.  M = 128 outputs (TMEM lanes), N = 64 maps (TMEM columns), K in tiles
// of 32 positions aligned to absolute ring positions.  FP32 accuracy from TF32
// tensor cores: operands are split into a TF32 high part and a TF32 residual
// and three MMAs (hi*hi + hi*lo + lo*hi) accumulate in FP32.
//
// belt_tile_prep_kernel writes, once per call, every belt ring of every map
// group as pre-split K x N tiles already in the canonical no-swizzle K-major
// layout (ring positions extended past both ends, so windows never wrap).  The
// contraction kernel then fetches each B tile with one 1-D TMA bulk copy
// (cp.async.bulk + mbarrier) issued before the threads build the matching A
// tile (weights split once per ring pair, 16-byte stores), so copy, build and
// the MMAs of the previous stage overlap.  After the last tile of a ring pair
// the partial accumulator is read back (tcgen05.ld) and Kahan-folded into FP32
// totals in shared memory, so FP32 rounding stays per ring pair.  Every
// mbarrier wait is bounded; on a timeout the kernel raises the device error
// flag, drains its pending operations and frees its tensor memory.
#include <cstdint>

#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_tc.cuh"

namespace ksc {
namespace {

constexpr int kM = 128;             // outputs per block (TMEM lanes)
constexpr int kN = 64;              // maps per group (TMEM columns)
constexpr int kKT = 32;             // positions per K tile (4 MMAs of K = 8)
constexpr int kThreads = 512;       // four threads per output row
constexpr int kParts = kThreads / kM;
constexpr int kTotStride = kN + 1;  // padded rows: conflict-free per-row access
constexpr int kTileB = kN * kKT;    // floats per B tile part (hi or lo)

struct Stage {  // one operand stage, canonical no-swizzle K-major tiles
    float a_hi[kM * kKT];
    float a_lo[kM * kKT];
    float b[2 * kTileB];  // hi then lo, copied as one block
};

using tc::mbar_wait;
using tc::mma_commit;
using tc::mma_tf32;
using tc::saddr;
using tc::split_tf32;

__host__ __device__ __forceinline__ int toff(int row, int k) { return tc::toff<kKT>(row, k); }

__device__ __forceinline__ uint64_t smem_desc(const void *p) { return tc::smem_desc<kKT>(p); }

// B tiles: for belt ring index qi, tile u (positions 32u - ext0 .. +31),
// map group g: kN x kKT hi floats then kN x kKT lo floats.
__global__ void belt_tile_prep_kernel(const ConvPlan P, const float *__restrict__ in,
                                      int n_maps, long long map_stride, int n_tiles, int ext0,
                                      int n_groups, float *__restrict__ ws) {
    const long long quads = (long long)(P.belt_hi - P.belt_lo + 1) * n_tiles * n_groups * kN *
                            (kKT / 4);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < quads;
         e += (long long)gridDim.x * blockDim.x) {
        const int kq = (int)(e % (kKT / 4));
        long long rest = e / (kKT / 4);
        const int n = (int)(rest % kN);
        rest /= kN;
        const int g = (int)(rest % n_groups);
        rest /= n_groups;
        const int u = (int)(rest % n_tiles);
        const int qi = (int)(rest / n_tiles);
        const DevRing Q = P.d_rings[P.belt_lo + qi];
        const int L = Q.len;
        const int map = g * kN + n;
        float hi[4], lo[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v = 0.0f;
            if (map < n_maps) {
                int p = (u * kKT + kq * 4 + c - ext0) % L;
                if (p < 0) p += L;
                v = __ldg(in + (long long)map * map_stride + Q.start + p);
            }
            split_tf32(v, &hi[c], &lo[c]);
        }
        float *blk = ws + (((long long)qi * n_tiles + u) * n_groups + g) * (2 * kTileB);
        const int o = toff(n, kq * 4);
        *reinterpret_cast<float4 *>(blk + o) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4 *>(blk + kTileB + o) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
conv_belt_mma_kernel(const ConvPlan P, const int2 *__restrict__ items, int n_items,
                     const float *__restrict__ ws, int n_tiles, int ext0, int n_groups,
                     float *__restrict__ out, int n_maps, long long map_stride, int w_cap,
                     int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Stage *stage = reinterpret_cast<Stage *>(smem_raw);  // 2 stages
    float *tot = reinterpret_cast<float *>(stage + 2);   // kM x kTotStride
    float *cmp = tot + kM * kTotStride;                  // Kahan compensation
    float *whi = cmp + kM * kTotStride;                  // w_cap split weights
    float *wlo = whi + w_cap;
    __shared__ __align__(8) uint64_t bfull[2], mdone[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (kM - 1), part = tid >> 7;  // output row; K-quad / column part
    constexpr int kCols = kN / kParts;                 // accumulator columns per thread
    const int g = blockIdx.y;  // map group
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(&tmem_base)),
                     "r"(kN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bfull[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mdone[b])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc::idesc_tf32(kM, kN);  // F32 += TF32 x TF32, K-major
    uint32_t ph_full[2] = {0u, 0u}, ph_done[2] = {0u, 0u};
    int pending[2] = {0, 0};
    int copy_b = -1;  // stage of the last bulk copy thread 0 issued and has not waited for
    bool ok = true;

    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        const int r = items[it].x, k0 = items[it].y;
        const DevRing R = P.d_rings[r];
        const int L = R.len;
        const int2 rg = P.d_range[r];
        const int q_lo = max(rg.x, P.belt_lo), q_hi = min(rg.y, P.belt_hi);
        const PairInfo *pinfo = P.d_pairs + P.d_pair_base[r] - rg.x;
        for (int n = part * kCols; n < (part + 1) * kCols; ++n) {
            tot[row * kTotStride + n] = 0.0f;
            cmp[row * kTotStride + n] = 0.0f;
        }
        int tcount = 0;
        for (int q = q_lo; q <= q_hi && ok; ++q) {
            const PairInfo pi = pinfo[q];
            if (pi.w < 0) continue;
            const DevRing Qr = P.d_rings[q];
            int lo = -pi.w, hi = pi.w;
            if (hi - lo + 1 >= L) {
                lo = -(L / 2);
                hi = lo + L - 1;
            }
            const int nd = hi - lo + 1;
            if (nd > w_cap) {  // never expected: the host sized w_cap for every pair
                if (tid == 0) atomicExch(err, KSC_ERR_DEVICE_BOUNDS);
                continue;
            }
            __syncthreads();  // previous readers of whi / wlo are done
            {
                const DF A = DF{pi.Ah, pi.Al}, B = DF{pi.Bh, pi.Bl};
                const DF c1 = DF{P.belt_c1h, P.belt_c1l};
                const int tdiff = R.phase - Qr.phase;
                for (int j = tid; j < nd; j += kThreads) {
                    const int D = lo + j;
                    const float mf = (float)(tdiff - 2 * D);
                    const float xh = mf * c1.h;
                    const float xl = fmaf(mf, c1.h, -xh) + mf * c1.l;
                    int ti;
                    float f;
                    float wv = 0.0f;
                    if (chord_to_table_padded(A, B, sin_df(xh, xl), P.nint2, &ti, &f))
                        wv = hermite(__ldg(&P.d_tab[min(ti, P.n_int)]), f);
                    split_tf32(wv, &whi[j], &wlo[j]);
                }
            }
            __syncthreads();
            // K tiles aligned to absolute positions: p in [P0, P1]
            const int P0 = (k0 + lo) & ~(kKT - 1);
            const int P1 = k0 + kM - 1 + hi;
            const int u0 = (P0 + ext0) / kKT, u1 = (P1 + ext0) / kKT;
            const float *blk0 = ws + (((long long)(q - P.belt_lo) * n_tiles) * n_groups + g) *
                                         (2 * kTileB);
            const long long ustride = (long long)n_groups * (2 * kTileB);
            const int base = P0 - k0 - lo;  // weight index of (row 0, column 0)
            for (int u = u0; u <= u1; ++u) {
                const int b = tcount & 1;
                if (pending[b]) {  // the MMAs that last read this stage are done
                    if (!mbar_wait(&mdone[b], ph_done[b])) s_abort = 1;
                    ph_done[b] ^= 1u;
                    pending[b] = 0;
                }
                Stage &S = stage[b];
                if (tid == 0 && !s_abort) {  // B tile: one bulk copy
                    const uint32_t bytes = 2u * kTileB * 4u;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     saddr(&bfull[b])),
                                 "r"(bytes)
                                 : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], "
                        "[%1], %2, [%3];" ::"r"(saddr(S.b)),
                        "l"(blk0 + (long long)u * ustride), "r"(bytes), "r"(saddr(&bfull[b]))
                        : "memory");
                    copy_b = b;
                }
                // A tile row `row`, K quads part, part + 4:
                // A[m][jj] = w[base + 32 (u - u0) + jj - m]
                {
                    const int m = row;
                    const int wi0 = base + kKT * (u - u0) - m;
#pragma unroll
                    for (int jj = 0; jj < (kKT / 4) / kParts; ++jj) {
                        const int jq = 4 * (part + kParts * jj);
                        float h[4], l[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int wi = wi0 + jq + c;
                            const bool in = wi >= 0 && wi < nd;
                            h[c] = in ? whi[wi] : 0.0f;
                            l[c] = in ? wlo[wi] : 0.0f;
                        }
                        const int o = toff(m, jq);
                        *reinterpret_cast<float4 *>(S.a_hi + o) = make_float4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<float4 *>(S.a_lo + o) = make_float4(l[0], l[1], l[2], l[3]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (s_abort) {  // uniform: read after the barrier
                    ok = false;
                    break;
                }
                if (tid == 0) {
                    copy_b = -1;
                    if (!mbar_wait(&bfull[b], ph_full[b])) {
                        s_abort = 1;
                    } else {
#pragma unroll
                        for (int s = 0; s < kKT / 8; ++s) {
                            const uint64_t ah = smem_desc(S.a_hi + s * 64);
                            const uint64_t al = smem_desc(S.a_lo + s * 64);
                            const uint64_t bh = smem_desc(S.b + s * 64);
                            const uint64_t bl = smem_desc(S.b + kTileB + s * 64);
                            const uint32_t first = (u == u0 && s == 0) ? 0u : 1u;
                            mma_tf32(tmem, ah, bh, idesc, first);
                            mma_tf32(tmem, ah, bl, idesc, 1u);
                            mma_tf32(tmem, al, bh, idesc, 1u);
                        }
                        mma_commit(&mdone[b]);
                    }
                }
                ph_full[b] ^= 1u;
                pending[b] = 1;
                ++tcount;
            }
            if (!ok) break;
            // drain: every MMA of this ring pair has completed
            for (int bb = 0; bb < 2; ++bb) {
                const int b = (tcount + bb) & 1;  // older stage first
                if (pending[b]) {
                    if (!mbar_wait(&mdone[b], ph_done[b])) s_abort = 1;
                    ph_done[b] ^= 1u;
                    pending[b] = 0;
                }
            }
            __syncthreads();
            if (s_abort) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // fold this ring pair's partial (row = TMEM lane, this thread's column
            // part) into the totals
#pragma unroll
            for (int c0 = part * kCols; c0 < (part + 1) * kCols; c0 += 16) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
                tc::tmem_ld16(ta, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int jv = 0; jv < 16; ++jv) {
                    float *s = tot + row * kTotStride + c0 + jv;
                    float *cc = cmp + row * kTotStride + c0 + jv;
                    const float y = __uint_as_float(v[jv]) - *cc;
                    const float tt = *s + y;
                    *cc = (tt - *s) - y;
                    *s = tt;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        if (!ok) break;
        const int k = k0 + row;
        if (k < L) {
            for (int n = part * kCols; n < (part + 1) * kCols && g * kN + n < n_maps; ++n)
                out[(long long)(g * kN + n) * map_stride + R.start + k] =
                    tot[row * kTotStride + n] * P.domega;
        }
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(err, KSC_ERR_TIMEOUT);
            if (copy_b >= 0) mbar_wait(&bfull[copy_b], ph_full[copy_b]);  // bulk copy in flight
        }
        for (int b = 0; b < 2; ++b) {  // bounded drain of MMAs still in flight
            if (pending[b]) mbar_wait(&mdone[b], ph_done[b]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kN));
}

} // namespace

int belt_mma_block() { return kM; }
int belt_mma_maps() { return kN; }

size_t belt_mma_smem(int w_cap) {
    return 2 * sizeof(Stage) + sizeof(float) * (2 * kM * kTotStride + 2 * (size_t)w_cap);
}

size_t belt_mma_workspace_floats(int n_belt, int n_tiles, int n_maps) {
    const int groups = (n_maps + kN - 1) / kN;
    return (size_t)n_belt * n_tiles * groups * 2 * kTileB;
}

cudaError_t launch_conv_belt_mma(const ConvPlan &p, const int2 *d_items, int n_items, int w_cap,
                                 int n_tiles, int ext0, float *d_ws, const float *d_in,
                                 float *d_out, int n_maps, long long map_stride, int *d_err,
                                 cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    const int groups = (n_maps + kN - 1) / kN;
    belt_tile_prep_kernel<<<4 * n_sm, 256, 0, st>>>(p, d_in, n_maps, map_stride, n_tiles, ext0,
                                                    groups, d_ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = belt_mma_smem(w_cap);
    e = cudaFuncSetAttribute(conv_belt_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = n_sm;  // one CTA per SM (shared memory, 64 TMEM columns each)
    if (blocks > n_items) blocks = n_items;
    dim3 grid(blocks, groups);
    conv_belt_mma_kernel<<<grid, kThreads, smem, st>>>(p, d_items, n_items, d_ws, n_tiles, ext0,
                                                       groups, d_out, n_maps, map_stride, w_cap,
                                                       d_err);
    return cudaGetLastError();
}

} // namespace ksc
