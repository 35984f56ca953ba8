// Real-space convolution, symmetric gather for rings outside the circulant
// belt path (polar caps, and belt rings whose disc reaches a cap).
//
// HEALPix RING geometry is invariant under a quarter turn about the polar axis
// (pixel k of a ring of L pixels maps to k + L/4) and under the north/south
// mirror z -> -z (ring r maps to ring 4n-2-r with the same pixel phases).  A
// pixel pair and its images under these eight symmetries have the same chord,
// so one kernel evaluation serves eight pairs:
//
//   out[r,   k + q L/4] += w * m[r',   k' + q L'/4]    q = 0..3
//   out[r_s, k + q L/4] += w * m[r'_s, k' + q L'/4]    (mirror images)
//
// One thread owns output position k of the first quarter of a northern ring r
// and produces its eight images (four on the equator ring, which is its own
// mirror).  Chord, window and table arithmetic are those of the general
// gather: d^2 = A + B sin^2(dphi/2) with FP64 ring-pair constants and the
// exact integer N for dphi; K_r from the cubic Hermite table (read through
// the L1 cache); per input ring FP32 partial sums, Kahan-folded into totals.
#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr int kThreads = 128;
constexpr int kRingChunk = 64;
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ float sin_taylor(float x) {
    const float x2 = x * x;
    float p = 1.6059043836821613e-10f;
    p = fmaf(p, x2, -2.5052108385441720e-08f);
    p = fmaf(p, x2, 2.7557319223985893e-06f);
    p = fmaf(p, x2, -1.9841269841269841e-04f);
    p = fmaf(p, x2, 8.3333333333333333e-03f);
    p = fmaf(p, x2, -1.6666666666666667e-01f);
    p = fmaf(p, x2, 1.0f);
    return x * p;
}

template <bool MIRROR>
__device__ __forceinline__ void sym_item(const ConvPlan &P, int r, int k, bool active,
                                         bool skip_belt_inputs, bool add, int band_lo,
                                         int band_hi, const float *__restrict__ m,
                                         float *__restrict__ o,
                                         float *sA, float *sB, float *sC, float *sHW, int *sL,
                                         int *sS, int *sSm, int *sT) {
    const int tid = threadIdx.x;
    const DevRing R = P.d_rings[r];
    const int L = R.len, Q4 = L / 4;
    const int2 rg = P.d_range[r];
    constexpr int NS = MIRROR ? 8 : 4;
    float sum[NS], comp[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) sum[i] = comp[i] = 0.0f;

    for (int q0 = rg.x; q0 <= rg.y; q0 += kRingChunk) {
        const int nq = min(kRingChunk, rg.y - q0 + 1);
        __syncthreads();
        if (tid < nq) {
            const int q = q0 + tid;
            const DevRing Q = P.d_rings[q];
            const double dz = R.z - Q.z;
            const double ds = (Q.z - R.z) * (Q.z + R.z) / (R.s + Q.s);
            const double A = dz * dz + ds * ds;
            const double ss = R.s * Q.s;
            float hw;
            if (skip_belt_inputs && q >= P.belt_lo && q <= P.belt_hi) {
                hw = -1.0f;
            } else if (A > (double)P.dc2 * (1.0 + 1e-6)) {
                hw = -1.0f;
            } else {
                const double cdp = (P.cos_cut - R.z * Q.z) / ss;
                double dphi = cdp <= -1.0 ? 4.0 * kPi : (cdp >= 1.0 ? 0.0 : acos(cdp));
                hw = (float)(dphi * Q.len / (2.0 * kPi)) + 1.0f;
            }
            sA[tid] = (float)A;
            sB[tid] = (float)(4.0 * ss);
            sC[tid] = (float)(kPi / (2.0 * (double)L * (double)Q.len));
            sHW[tid] = hw;
            sL[tid] = Q.len;
            sS[tid] = Q.start;
            sSm[tid] = P.d_rings[P.nrings - 1 - q].start;
            sT[tid] = Q.phase;
        }
        __syncthreads();
        if (!active) continue;
        for (int qi = 0; qi < nq; ++qi) {
            const float hw = sHW[qi];
            if (hw < 0.0f) continue;
            const int L2 = sL[qi], Q2 = L2 / 4;
            const long long num = (long long)(2 * k + R.phase) * L2 - (long long)sT[qi] * L;
            const float kc = (float)num / (float)(2 * L);
            int klo = (int)floorf(kc - hw), khi = (int)ceilf(kc + hw);
            if (2.0f * hw + 1.0f >= (float)L2 || khi - klo + 1 >= L2) {
                klo = (int)floorf(kc) - L2 / 2;
                khi = klo + L2 - 1;
            }
            int N = (int)(num - 2LL * klo * L);
            int idx = klo % L2;
            if (idx < 0) idx += L2;
            const float A = sA[qi], B = sB[qi], cs = sC[qi];
            const float *mn = m + sS[qi];
            const float *ms = m + sSm[qi];
            float part[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) part[i] = 0.0f;
            for (int kk = klo; kk <= khi; ++kk) {
                const float sn = sin_taylor((float)N * cs);
                const float d2 = fmaf(B, sn * sn, A);
                if (d2 <= P.dc2) {
                    const float u = sqrtf(d2) * P.inv_h;
                    const int i = min((int)u, P.n_int - 1);
                    const float f = u - (float)i;
                    const float4 c = __ldg(&P.d_tab[i]);
                    const float w = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
                    int j = idx;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        part[qq] = fmaf(w, __ldg(mn + j), part[qq]);
                        if constexpr (MIRROR) part[4 + qq] = fmaf(w, __ldg(ms + j), part[4 + qq]);
                        j += Q2;
                        if (j >= L2) j -= L2;
                    }
                }
                N -= 2 * L;
                if (++idx == L2) idx = 0;
            }
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                const float y = part[i] - comp[i];
                const float t = sum[i] + y;
                comp[i] = (t - sum[i]) - y;
                sum[i] = t;
            }
        }
    }
    if (active) {
        const int rs = P.nrings - 1 - r;
        const int start_s = P.d_rings[rs].start;
        const bool wn = r >= band_lo && r <= band_hi;
        const bool ws = MIRROR && rs >= band_lo && rs <= band_hi;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int kq = k + qq * Q4;
            if (wn) {
                if (add) o[R.start + kq] += sum[qq] * P.domega;
                else o[R.start + kq] = sum[qq] * P.domega;
            }
            if constexpr (MIRROR) {
                if (ws) {
                    if (add) o[start_s + kq] += sum[4 + qq] * P.domega;
                    else o[start_s + kq] = sum[4 + qq] * P.domega;
                }
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads)
conv_sym_kernel(const ConvPlan P, const WorkItem *__restrict__ items, int n_items,
                const float *__restrict__ in, float *__restrict__ out, long long map_stride,
                int belt_split, int band_lo, int band_hi) {
    __shared__ float sA[kRingChunk], sB[kRingChunk], sC[kRingChunk], sHW[kRingChunk];
    __shared__ int sL[kRingChunk], sS[kRingChunk], sSm[kRingChunk], sT[kRingChunk];
    const float *m = in + (long long)blockIdx.y * map_stride;
    float *o = out + (long long)blockIdx.y * map_stride;
    const int eq = (P.nrings - 1) / 2;  // the equator ring, its own mirror image
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const WorkItem w = items[it];
        const int L = P.d_rings[w.ring].len;
        const int k = w.k0 + threadIdx.x;
        const bool active = k < L / 4;
        const bool belt = w.ring >= P.belt_lo && w.ring <= P.belt_hi;
        const bool add = belt_split && belt;
        if (w.ring == eq)
            sym_item<false>(P, w.ring, k, active, add, add, band_lo, band_hi, m, o, sA, sB, sC,
                            sHW, sL, sS, sSm, sT);
        else
            sym_item<true>(P, w.ring, k, active, add, add, band_lo, band_hi, m, o, sA, sB, sC,
                           sHW, sL, sS, sSm, sT);
    }
}

} // namespace

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
