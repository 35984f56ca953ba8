// Real-space convolution, general ring-pair gather (Sec. 1-2; Fig. 1 GPU half):
//
//   out_i = (4 pi / Npix) sum_{j: theta_ij <= theta_cut} K_r(theta_ij) m_j
//
// One thread owns one output pixel.  Input rings within theta_cut of the
// output ring are visited in chunks; per (output ring, input ring) pair the
// block precomputes in shared memory, in FP64 and rounded once to FP32,
//   A = (z - z')^2 + (s - s')^2,   B = 4 s s',
// so that the squared chord of any pixel pair of the two rings is
//   d^2 = A + B sin^2(dphi / 2)
// with every term non-negative (no cancellation near theta = 0).  dphi / 2 is
// N * pi / (2 L L') for the exact integer N = (2k + t) L' - (2k' + t') L
// (pixel k of a ring of L pixels sits at phi = (2k + t) pi / L), so no pixel
// coordinate is ever rounded.  sin is its Taylor series to x^13, accurate to
// FP32 rounding on |x| <= pi/2.  K_r(d) comes from the cubic Hermite table in
// shared memory; each input ring's FP32 partial sum is folded into the pixel
// total with Kahan compensation.
#include "ksc_device.cuh"
#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr int kThreads = 256;
constexpr int kRingChunk = 128;


template <bool COUNT>
__global__ void __launch_bounds__(kThreads)
conv_general_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                    const float *__restrict__ in, float *__restrict__ out,
                    long long map_stride, int belt_split,
                    unsigned long long *__restrict__ count) {
    extern __shared__ float4 s_tab[];
    __shared__ DF sA[kRingChunk], sB[kRingChunk], sC[kRingChunk];
    __shared__ float sHW[kRingChunk];
    __shared__ int sL[kRingChunk], sS[kRingChunk], sT[kRingChunk];

    const int tid = threadIdx.x;
    if (!COUNT)
        for (int i = tid; i < P.n_int; i += kThreads) s_tab[i] = P.d_tab[i];

    const float *m = in + (long long)blockIdx.y * map_stride;
    float *o = out + (long long)blockIdx.y * map_stride;
    unsigned long long cnt = 0;

    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const DevRing R = P.d_rings[w.ring];
        const int L = R.len;
        const int k = w.k0 + tid;
        const bool active = k < L;
        const int2 rg = P.d_range[w.ring];
        // belt output ring with the belt kernel in use: cap input rings only
        const bool add = !COUNT && belt_split && w.ring >= P.belt_lo && w.ring <= P.belt_hi;
        float sum = 0.0f, comp = 0.0f;

        for (int q0 = rg.x; q0 <= rg.y; q0 += kRingChunk) {
            const int nq = min(kRingChunk, rg.y - q0 + 1);
            __syncthreads();
            if (tid < nq) {
                const int q = q0 + tid;
                const DevRing Q = P.d_rings[q];
                const PairInfo pi = P.d_pairs[P.d_pair_base[w.ring] + (q - rg.x)];
                float hw;
                const bool bb = w.ring >= P.belt_lo && w.ring <= P.belt_hi &&
                                q >= P.belt_lo && q <= P.belt_hi;
                if ((add && bb) || (COUNT && belt_split == 1 && !bb) ||
                    (COUNT && belt_split == 2 && bb)) {
                    // belt-belt pair done by the circulant kernel, or a pair
                    // outside the class being counted
                    hw = -1.0f;
                } else {
                    hw = pi.hw;
                }
                sA[tid] = DF{pi.Ah, pi.Al};
                sB[tid] = DF{pi.Bh, pi.Bl};
                sC[tid] = DF{pi.ch, pi.cl};
                sHW[tid] = hw;
                sL[tid] = Q.len;
                sS[tid] = Q.start;
                sT[tid] = Q.phase;
            }
            __syncthreads();
            if (!active) continue;
            for (int qi = 0; qi < nq; ++qi) {
                const float hw = sHW[qi];
                if (hw < 0.0f) continue;
                const int L2 = sL[qi];
                const long long num = (long long)(2 * k + R.phase) * L2 - (long long)sT[qi] * L;
                const float kc = (float)num / (float)(2 * L);
                int klo = (int)floorf(kc - hw), khi = (int)ceilf(kc + hw);
                if (2.0f * hw + 1.0f >= (float)L2 || khi - klo + 1 >= L2) {
                    // the window covers the ring: every pixel exactly once,
                    // centred so that |dphi| <= pi (1 + 2/L2)
                    klo = (int)floorf(kc) - L2 / 2;
                    khi = klo + L2 - 1;
                }
                int N = (int)(num - 2LL * klo * L);
                int idx = klo % L2;
                if (idx < 0) idx += L2;
                const DF A = sA[qi], B = sB[qi], cs = sC[qi];
                const float *mr = m + sS[qi];
                // blocks of 32 window steps, each Kahan-folded into the total
                for (int kb0 = klo; kb0 <= khi; kb0 += 32) {
                    const int kend = min(kb0 + 31, khi);
                    float part = 0.0f;
                    for (int kk = kb0; kk <= kend; ++kk) {
                        const float Nf = (float)N;
                        const float xh = Nf * cs.h;
                        const float xl = fmaf(Nf, cs.h, -xh) + Nf * cs.l;
                        int ti;
                        float f;
                        if (chord_to_table(A, B, sin_df(xh, xl), P.nint2, P.n_int, &ti, &f)) {
                            if (COUNT) {
                                ++cnt;
                            } else {
                                part = fmaf(hermite(s_tab[ti], f), __ldg(mr + idx), part);
                            }
                        }
                        N -= 2 * L;
                        if (++idx == L2) idx = 0;
                    }
                    const float y = part - comp;
                    const float t = sum + y;
                    comp = (t - sum) - y;
                    sum = t;
                }
            }
        }
        if (!COUNT && active) {
            if (add)
                o[R.start + k] += sum * P.domega;
            else
                o[R.start + k] = sum * P.domega;
        }
    }
    if (COUNT) {
        // block reduction of the pair counts
        __shared__ unsigned long long s_cnt[kThreads / 32];
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, off);
        if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
        __syncthreads();
        if (tid == 0) {
            unsigned long long t = 0;
            for (int i = 0; i < kThreads / 32; ++i) t += s_cnt[i];
            atomicAdd(count, t);
        }
    }
}

} // namespace

cudaError_t launch_conv_general(const ConvPlan &p, const WorkItem *d_items, int n_items,
                                const float *d_in, float *d_out, int n_maps,
                                long long map_stride, int belt_split,
                                unsigned long long *d_count, cudaStream_t st) {
    if (n_items <= 0 || n_maps <= 0) return cudaSuccess;
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    const bool count = d_count != nullptr;
    const size_t smem = count ? 0 : sizeof(float4) * (size_t)p.n_int;
    int per_sm = 0;
    cudaError_t e;
    if (count) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_general_kernel<true>,
                                                          kThreads, smem);
    } else {
        e = cudaFuncSetAttribute(conv_general_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, conv_general_kernel<false>,
                                                          kThreads, smem);
    }
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int blocks = n_sm * per_sm;
    if (blocks > n_items) blocks = n_items;
    dim3 grid(blocks, n_maps);
    if (count)
        conv_general_kernel<true><<<grid, kThreads, smem, st>>>(p, d_items, n_items, d_in, d_out,
                                                               map_stride, belt_split, d_count);
    else
        conv_general_kernel<false><<<grid, kThreads, smem, st>>>(p, d_items, n_items, d_in, d_out,
                                                                map_stride, belt_split, d_count);
    return cudaGetLastError();
}

} // namespace ksc
