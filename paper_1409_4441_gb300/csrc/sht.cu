// The harmonic half of the split convolution on the GPU (Fig. 1's CPU half; an
// option of this library): spherical-harmonic synthesis and analysis of HEALPix
// RING maps up to l_max, m <= l_max, real fields, declared in include/ksconv.h.
//
//   synthesis  m_p = sum_l a_l0 lambda_l0(z) + 2 Re sum_{m>0} G_m(z) e^{i m phi},
//              G_m(z) = sum_l a_lm lambda_lm(z);
//   analysis   a_lm = (4 pi / Npix) sum_rings lambda_lm(z) F_m(ring),
//              F_m = sum_k m_k e^{-i m phi_k}.
//
// lambda_lm are the normalised associated Legendre functions without the
// Condon-Shortley phase, from their three-term recurrence in l at fixed m
// (lambda_mm = sqrt((2m+1)/4pi prod_{k<=m} (2k-1)/2k) sin^m theta; lambda_{m+1,m}
// = sqrt(2m+3) z lambda_mm; lambda_lm = A_l (z lambda_{l-1,m} - lambda_{l-2,m} /
// A_{l-1}), A_l = sqrt((4l^2-1)/(l^2-m^2))), in FP64 with a scale exponent:
// near the poles sin^m theta underflows any floating format, so values are
// carried as v 2^(600 e) and summed only once e reaches 0 (while e < 0 the true
// value is below 2^-300).  North and south rings share |z| (lambda_lm(-z) =
// (-1)^(l+m) lambda_lm(z)), so each recurrence serves a ring pair through its
// even and odd partial sums.
//
// The ring sums over m (synthesis) and over pixels (analysis) are direct sums in
// FP32 restricted to m <= l_max: pixel k of a ring of L pixels with phase flag t
// sits at phi_k = pi (2k + t) / L, so m phi_k = pi J / L with the exact integer
// J = m (2k + t) mod 2L; the twiddles advance by one complex product per step
// and are re-anchored from the exact J every 8 steps (the products' rounding
// drifts by about one FP32 ulp per step in between).
#include <cstdint>

#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kAnchor = 8;        // twiddle steps between exact re-anchors
constexpr double kScale = 600.0;  // log2 of one scale step of the recurrence

__host__ __device__ inline long long n_alm(int lmax) {
    return (long long)(lmax + 1) * (lmax + 2) / 2;
}
__host__ __device__ inline long long alm_base(int lmax, int m) {  // index(0, m)
    return (long long)m * (2 * lmax + 1 - m) / 2;
}

// Ring r (0-based) of nside n: z, sin theta (FP64, 1 - z kept exact near the
// north pole), pixel count, first pixel, phase flag.
struct ShtRing {
    double z, s;
    int len, start, t;
};
__device__ inline ShtRing sht_ring(int n, int r) {
    const long long i = r + 1;
    const double nn = (double)n;
    ShtRing g;
    double omz, opz;
    if (i < n) {
        omz = (double)(i * i) / (3.0 * nn * nn);
        g.z = 1.0 - omz;
        opz = 1.0 + g.z;
        g.len = (int)(4 * i);
        g.start = (int)(2 * i * (i - 1));
        g.t = 1;
    } else if (i <= 3LL * n) {
        g.z = (double)(4LL * n - 2 * i) / (3.0 * nn);
        omz = 1.0 - g.z;
        opz = 1.0 + g.z;
        g.len = 4 * n;
        g.start = (int)(2LL * n * (n - 1) + 4LL * n * (i - n));
        g.t = ((i - n) % 2 == 0) ? 1 : 0;
    } else {
        const long long ip = 4LL * n - i;
        opz = (double)(ip * ip) / (3.0 * nn * nn);
        g.z = opz - 1.0;
        omz = 1.0 - g.z;
        g.len = (int)(4 * ip);
        g.start = (int)(12LL * n * n - 2 * ip * (ip + 1));
        g.t = 1;
    }
    g.s = sqrt(omz * opz);
    return g;
}

// Start of the recurrence at l = m: lambda_mm = v 2^(600 e), v in [2^-300, 2^300).
__device__ inline void lambda_mm(int m, double s, double *v, int *e) {
    // log2 lambda_mm = 1/2 log2((2m+1)/4pi) + 1/2 log2((2m)! / (4^m m!^2)) + m log2 s
    const double lg = 0.5 * log2((2.0 * m + 1.0) / (4.0 * kPi)) +
                      0.5 * (lgamma(2.0 * m + 1.0) - 2.0 * lgamma(m + 1.0)) / log(2.0) - m +
                      (m > 0 ? m * log2(s) : 0.0);
    int ee = (int)floor((lg + 300.0) / kScale);
    if (ee > 0) ee = 0;
    *e = ee;
    *v = exp2(lg - kScale * ee);
}

// The recurrence coefficients of order m in shared memory: A[l] (l = m+1..lmax)
// and B[l] = 1 / A[l-1] (l = m+2..lmax).
__device__ inline void build_coeffs(int m, int lmax, double *A, double *B) {
    for (int l = m + 1 + threadIdx.x; l <= lmax; l += blockDim.x) {
        const double ll = (double)l, mm = (double)m;
        A[l] = sqrt((4.0 * ll * ll - 1.0) / ((ll - mm) * (ll + mm)));
        if (l >= m + 2) {
            const double l1 = ll - 1.0;
            B[l] = sqrt((l1 - mm) * (l1 + mm) / (4.0 * l1 * l1 - 1.0));
        }
    }
}

// Synthesis, Legendre part: G[ring][m] = sum_l a_lm lambda_lm(z_ring) for every
// northern ring (and its southern mirror) of the block's range and order m =
// blockIdx.y.  One thread per northern ring.
__global__ void __launch_bounds__(128)
sht_leg_synth(int nside, int lmax, const double2 *__restrict__ alm, float2 *__restrict__ G) {
    extern __shared__ double coef[];
    const int m = blockIdx.y;
    double *A = coef, *B = coef + (lmax + 1);
    build_coeffs(m, lmax, A, B);
    __syncthreads();
    const int nnorth = 2 * nside, nr = 4 * nside - 1;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nnorth) return;
    const ShtRing g = sht_ring(nside, r);
    const double2 *a = alm + alm_base(lmax, m);
    double v2 = 0.0, v1;
    int e;
    lambda_mm(m, g.s, &v1, &e);
    double er = 0.0, ei = 0.0, orr = 0.0, oi = 0.0;  // even / odd (l - m) sums
    if (e == 0) {
        const double2 c = __ldg(a + m);
        er = v1 * c.x;
        ei = v1 * c.y;
    }
    const double z = g.z;
    for (int l = m + 1; l <= lmax; ++l) {
        const double v = A[l] * (z * v1 - (l >= m + 2 ? B[l] * v2 : 0.0));
        v2 = v1;
        v1 = v;
        if (e < 0) {
            if (fabs(v1) >= 0x1p300) {  // one scale step up
                v1 *= 0x1p-600;
                v2 *= 0x1p-600;
                ++e;
            }
            if (e < 0) continue;
        }
        const double2 c = __ldg(a + l);
        if ((l - m) & 1) {
            orr = fma(v1, c.x, orr);
            oi = fma(v1, c.y, oi);
        } else {
            er = fma(v1, c.x, er);
            ei = fma(v1, c.y, ei);
        }
    }
    const long long stride = lmax + 1;
    G[(long long)r * stride + m] = make_float2((float)(er + orr), (float)(ei + oi));
    const int rs = nr - 1 - r;
    if (rs != r) G[(long long)rs * stride + m] = make_float2((float)(er - orr), (float)(ei - oi));
}

// e^{i pi J / L} for the exact integer J = a b mod 2L (a, b >= 0), to about one
// FP32 ulp: J / L = hi + lo with hi the rounded quotient and lo = (J - hi L) / L
// (the remainder exact by the fused multiply-add), J folded into [-L, L); the
// rounding of hi is undone to first order, e^{i pi lo} = 1 + i pi lo.
__device__ inline float2 twiddle(long long a, long long b, int L) {
    long long J = (a % (2LL * L)) * (b % (2LL * L)) % (2LL * L);
    if (J >= L) J -= 2LL * L;
    const float fj = (float)J, fl = (float)L;  // exact: |J|, L <= 2^15
    const float hi = fj / fl;
    const float lo = fmaf(-hi, fl, fj) / fl;
    float sn, cs;
    sincospif(hi, &sn, &cs);
    const float d = 3.14159265f * lo;
    return make_float2(fmaf(-sn, d, cs), fmaf(cs, d, sn));
}

__device__ inline float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Synthesis, ring part: for northern ring r = blockIdx.x and its mirror, pixel k
// gets sum_m w_m Re(G_m e^{i m phi_k}) (w_0 = 1, else 2); add != 0 adds it to
// the map.  G of both rings staged in shared memory (pre-weighted).
__global__ void __launch_bounds__(256)
sht_dft_synth(int nside, int lmax, const float2 *__restrict__ G, float *__restrict__ map,
              int add) {
    extern __shared__ float2 gs[];  // [2][lmax + 1]
    const int r = blockIdx.x, nr = 4 * nside - 1, rs = nr - 1 - r;
    const bool mirror = rs != r;
    const long long stride = lmax + 1;
    for (int m = threadIdx.x; m <= lmax; m += blockDim.x) {
        const float w = m == 0 ? 1.0f : 2.0f;
        const float2 a = G[(long long)r * stride + m];
        gs[m] = make_float2(w * a.x, w * a.y);
        const float2 b = mirror ? G[(long long)rs * stride + m] : make_float2(0.0f, 0.0f);
        gs[stride + m] = make_float2(w * b.x, w * b.y);
    }
    __syncthreads();
    const ShtRing g = sht_ring(nside, r);
    const int L = g.len;
    const ShtRing h = sht_ring(nside, rs);
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const long long q = 2LL * k + g.t;  // m phi_k = pi m q / L
        const float2 step = twiddle(1, q, L);
        float sn = 0.0f, cn = 0.0f, ss = 0.0f, cc = 0.0f;  // sums and compensations
        for (int m0 = 0; m0 <= lmax; m0 += kAnchor) {
            float2 w = twiddle(m0, q, L);
            float pn = 0.0f, ps = 0.0f;
            const int m1 = min(m0 + kAnchor, lmax + 1);
            for (int m = m0; m < m1; ++m) {
                const float2 a = gs[m], b = gs[stride + m];
                pn = fmaf(a.x, w.x, fmaf(-a.y, w.y, pn));
                ps = fmaf(b.x, w.x, fmaf(-b.y, w.y, ps));
                w = cmul(w, step);
            }
            // compensated accumulation of the chunk partials
            float y = pn - cn, t2 = sn + y;
            cn = (t2 - sn) - y;
            sn = t2;
            y = ps - cc;
            t2 = ss + y;
            cc = (t2 - ss) - y;
            ss = t2;
        }
        float *on = map + g.start + k;
        if (add) *on += sn; else *on = sn;
        if (mirror) {
            float *os = map + h.start + k;
            if (add) *os += ss; else *os = ss;
        }
    }
}

constexpr int kAnalChunk = 4096;  // pixels of each ring staged per pass

// Analysis, ring part: F[ring][m] = sum_k m_k e^{-i m phi_k} for northern ring r =
// blockIdx.x and its mirror, every m <= lmax (threads over m).  Pixels staged in
// shared memory in chunks; FP32 partials over 64 pixels summed in FP64.
__global__ void __launch_bounds__(256)
sht_dft_anal(int nside, int lmax, const float *__restrict__ map, float2 *__restrict__ F) {
    __shared__ float2 px[kAnalChunk];  // (north, south) pixel values
    const int r = blockIdx.x, nr = 4 * nside - 1, rs = nr - 1 - r;
    const bool mirror = rs != r;
    const ShtRing g = sht_ring(nside, r);
    const ShtRing h = sht_ring(nside, rs);
    const int L = g.len;
    const long long stride = lmax + 1;
    const int per = (lmax + blockDim.x) / blockDim.x;  // orders per thread
    for (int j = 0; j < per; ++j) {
        const int m = threadIdx.x + j * blockDim.x;
        const bool live = m <= lmax;
        // step e^{-i m 2 pi / L}; the pixels of the chunk are k0 .. k0 + n - 1
        const float2 st = live ? twiddle(m, 2, L) : make_float2(1.0f, 0.0f);
        const float2 step = make_float2(st.x, -st.y);
        double fnr = 0.0, fni = 0.0, fsr = 0.0, fsi = 0.0;
        for (int k0 = 0; k0 < L; k0 += kAnalChunk) {
            const int n = min(kAnalChunk, L - k0);
            __syncthreads();
            for (int k = threadIdx.x; k < n; k += blockDim.x)
                px[k] = make_float2(map[g.start + k0 + k], mirror ? map[h.start + k0 + k] : 0.0f);
            __syncthreads();
            if (!live) continue;
            for (int b0 = 0; b0 < n; b0 += 64) {
                float pnr = 0.0f, pni = 0.0f, psr = 0.0f, psi = 0.0f;
                const int b1 = min(b0 + 64, n);
                for (int a0 = b0; a0 < b1; a0 += kAnchor) {
                    const float2 c = twiddle(m, 2LL * (k0 + a0) + g.t, L);
                    float2 w = make_float2(c.x, -c.y);  // e^{-i m phi_k}
                    const int a1 = min(a0 + kAnchor, b1);
                    for (int k = a0; k < a1; ++k) {
                        const float2 v = px[k];
                        pnr = fmaf(v.x, w.x, pnr);
                        pni = fmaf(v.x, w.y, pni);
                        psr = fmaf(v.y, w.x, psr);
                        psi = fmaf(v.y, w.y, psi);
                        w = cmul(w, step);
                    }
                }
                fnr += pnr;
                fni += pni;
                fsr += psr;
                fsi += psi;
            }
        }
        if (live) {
            F[(long long)r * stride + m] = make_float2((float)fnr, (float)fni);
            if (mirror) F[(long long)rs * stride + m] = make_float2((float)fsr, (float)fsi);
        }
    }
}

// Analysis, Legendre part: alm[l, m] += c K_l sum_rings lambda_lm(z) F_m for the
// northern rings of the block's range (one per thread, with their mirrors) and
// order m = blockIdx.y; c = 4 pi / Npix, K_l = kl[l] (kl NULL: 1).  Each warp
// sums its 32 rings by shuffles, lane 0 adds to alm (zeroed by the caller).
__global__ void __launch_bounds__(128)
sht_leg_anal(int nside, int lmax, const float2 *__restrict__ F, const double *__restrict__ kl,
             double c, double2 *__restrict__ alm) {
    extern __shared__ double coef[];
    const int m = blockIdx.y;
    double *A = coef, *B = coef + (lmax + 1);
    build_coeffs(m, lmax, A, B);
    __syncthreads();
    const int nnorth = 2 * nside, nr = 4 * nside - 1;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = r < nnorth;
    const int lane = threadIdx.x & 31;
    const long long stride = lmax + 1;
    double sr = 0.0, si = 0.0, dr = 0.0, di = 0.0, z = 0.0, v1 = 0.0, v2 = 0.0;
    int e = -1;
    if (live) {
        const ShtRing g = sht_ring(nside, r);
        z = g.z;
        const int rs = nr - 1 - r;
        const float2 fn = F[(long long)r * stride + m];
        const float2 fs = rs != r ? F[(long long)rs * stride + m] : make_float2(0.0f, 0.0f);
        sr = (double)fn.x + fs.x;  // even l - m: lambda(z) = lambda(-z)
        si = (double)fn.y + fs.y;
        dr = (double)fn.x - fs.x;  // odd l - m
        di = (double)fn.y - fs.y;
        lambda_mm(m, g.s, &v1, &e);
    }
    double2 *a = alm + alm_base(lmax, m);
    for (int l = m; l <= lmax; ++l) {
        if (l > m) {
            const double v = A[l] * (z * v1 - (l >= m + 2 ? B[l] * v2 : 0.0));
            v2 = v1;
            v1 = v;
            if (e < 0 && fabs(v1) >= 0x1p300) {
                v1 *= 0x1p-600;
                v2 *= 0x1p-600;
                ++e;
            }
        }
        const bool on = live && e == 0;
        if (!__any_sync(0xffffffffu, on)) continue;
        const bool odd = (l - m) & 1;
        double xr = on ? v1 * (odd ? dr : sr) : 0.0;
        double xi = on ? v1 * (odd ? di : si) : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            xr += __shfl_down_sync(0xffffffffu, xr, o);
            xi += __shfl_down_sync(0xffffffffu, xi, o);
        }
        if (lane == 0) {
            const double w = c * (kl ? kl[l] : 1.0);
            atomicAdd(&a[l].x, w * xr);
            atomicAdd(&a[l].y, w * xi);
        }
    }
}

// Dynamic shared memory of the Legendre kernels (A and B tables) and of the
// synthesis ring kernel (two rings' G): the same size; above 48 kB the kernels
// are opted in for it.
cudaError_t leg_smem(int lmax, size_t *bytes) {
    *bytes = sizeof(double) * 2 * (size_t)(lmax + 1);
    if (*bytes <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(sht_leg_synth,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sht_leg_anal, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)*bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sht_dft_synth, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)*bytes);
    return e;
}

}  // namespace

// alm (device, n_alm(lmax) complex) -> map (device FP32); add != 0 adds.
cudaError_t sht_synthesis(int nside, int lmax, const double2 *d_alm, float *d_map, int add,
                          cudaStream_t st) {
    size_t cs = 0;
    cudaError_t e = leg_smem(lmax, &cs);
    if (e != cudaSuccess) return e;
    const int nr = 4 * nside - 1, nnorth = 2 * nside;
    float2 *G = nullptr;
    if ((e = cudaMallocAsync(&G, sizeof(float2) * (size_t)nr * (lmax + 1), st)) != cudaSuccess)
        return e;
    dim3 grid((nnorth + 127) / 128, lmax + 1);
    sht_leg_synth<<<grid, 128, cs, st>>>(nside, lmax, d_alm, G);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        sht_dft_synth<<<nnorth, 256, cs, st>>>(
            nside, lmax, G, d_map, add);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(G, st);
    return e != cudaSuccess ? e : f;
}

// map (device FP32) -> alm (device, n_alm(lmax) complex), each a_lm scaled by kl[l]
// when kl (device, lmax + 1 doubles) is given.
cudaError_t sht_analysis(int nside, int lmax, const float *d_map, const double *d_kl,
                         double2 *d_alm, cudaStream_t st) {
    size_t cs = 0;
    cudaError_t e = leg_smem(lmax, &cs);
    if (e != cudaSuccess) return e;
    const int nr = 4 * nside - 1, nnorth = 2 * nside;
    float2 *F = nullptr;
    if ((e = cudaMallocAsync(&F, sizeof(float2) * (size_t)nr * (lmax + 1), st)) != cudaSuccess)
        return e;
    e = cudaMemsetAsync(d_alm, 0, sizeof(double2) * (size_t)n_alm(lmax), st);
    if (e == cudaSuccess) {
        sht_dft_anal<<<nnorth, 256, 0, st>>>(nside, lmax, d_map, F);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const double c = 4.0 * kPi / (12.0 * (double)nside * (double)nside);
        dim3 grid((nnorth + 127) / 128, lmax + 1);
        sht_leg_anal<<<grid, 128, cs, st>>>(nside, lmax, F, d_kl, c, d_alm);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(F, st);
    return e != cudaSuccess ? e : f;
}

long long sht_n_alm(int lmax) { return n_alm(lmax); }

}  // namespace ksc

namespace {

int sht_fail(int code, const char *msg) {
    ksc::set_last_error(msg);
    return code;
}

int sht_cuda(cudaError_t e, const char *what) {
    return sht_fail(e == cudaErrorMemoryAllocation ? KSC_ERR_NOMEM : KSC_ERR_CUDA, what);
}

int sht_args(int nside, int lmax) {
    if (nside < 1 || nside > 8192 || (nside & (nside - 1)))
        return sht_fail(KSC_ERR_ARG, "nside must be a power of two <= 8192");
    if (lmax < 0 || lmax > 4 * nside || lmax > 8191)
        return sht_fail(KSC_ERR_ARG, "lmax outside 0..min(4 nside, 8191)");
    return KSC_OK;
}

}  // namespace

extern "C" {

int ksc_sht_alm2map(int nside, int lmax, const double *d_alm, float *d_map, void *stream) {
    ksc::NvtxRange range("ksc_sht_alm2map");
    int rc = sht_args(nside, lmax);
    if (rc) return rc;
    if (!d_alm || !d_map) return sht_fail(KSC_ERR_ARG, "null pointer");
    const cudaError_t e = ksc::sht_synthesis(nside, lmax, (const double2 *)d_alm, d_map, 0,
                                             (cudaStream_t)stream);
    return e == cudaSuccess ? KSC_OK : sht_cuda(e, "spherical-harmonic synthesis");
}

int ksc_sht_map2alm(int nside, int lmax, const float *d_map, double *d_alm, void *stream) {
    ksc::NvtxRange range("ksc_sht_map2alm");
    int rc = sht_args(nside, lmax);
    if (rc) return rc;
    if (!d_alm || !d_map) return sht_fail(KSC_ERR_ARG, "null pointer");
    const cudaError_t e = ksc::sht_analysis(nside, lmax, d_map, nullptr, (double2 *)d_alm,
                                            (cudaStream_t)stream);
    return e == cudaSuccess ? KSC_OK : sht_cuda(e, "spherical-harmonic analysis");
}

int ksc_conv_harmonic(const ksc_split *s, const float *d_in, float *d_out, int add,
                      void *stream) {
    ksc::NvtxRange range("ksc_conv_harmonic");
    if (!s || !d_in || !d_out) return sht_fail(KSC_ERR_ARG, "null argument");
    const int lc = s->l_cut;
    if (lc < 0 || (int)s->k_harm.size() < lc + 1)
        return sht_fail(KSC_ERR_ARG, "the split has no harmonic part");
    int rc = sht_args(s->nside, lc);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *kl = nullptr;
    double2 *alm = nullptr;
    cudaError_t e = cudaMallocAsync(&kl, sizeof(double) * (size_t)(lc + 1), st);
    if (e == cudaSuccess)
        e = cudaMallocAsync(&alm, sizeof(double2) * (size_t)ksc::sht_n_alm(lc), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(kl, s->k_harm.data(), sizeof(double) * (size_t)(lc + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = ksc::sht_analysis(s->nside, lc, d_in, kl, alm, st);
    if (e == cudaSuccess) e = ksc::sht_synthesis(s->nside, lc, alm, d_out, add ? 1 : 0, st);
    if (kl) cudaFreeAsync(kl, st);
    if (alm) cudaFreeAsync(alm, st);
    return e == cudaSuccess ? KSC_OK : sht_cuda(e, "harmonic half");
}

}  // extern "C"
