/*
 * FP64 CPU oracle for the compact-kernel spherical convolution (arXiv:1409.4441).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA library: geometry, Legendre
 * sums, the convolution and the spherical-harmonic transform are all written
 * out here again, plainly, in double precision, without blocking or reuse.
 *
 * Contents
 *   - HEALPix RING geometry (Gorski et al. 2005, cited by the paper in Sec. 2
 *     for its nside = 2048 data set).
 *   - Legendre sums K(z) = sum_l (2l+1)/(4 pi) c_l P_l(z) and dK/dz: the
 *     Legendre transformation operator P_{l theta} of Eq. 1, in the
 *     normalisation where c_0 = 1 means a unit-integral kernel.
 *   - All-pairs brute-force real-space convolution: every output pixel sums
 *     K(theta_ij) m_j (4 pi / Npix) over every input pixel with
 *     theta_ij <= theta_cut (the real-space half of Fig. 1, Sec. 2).
 *   - The Legendre stage of a ring-based spherical-harmonic transform
 *     (analysis and synthesis), i.e. the harmonic half of Fig. 1; the
 *     phi-direction sums are done by the Python glue with an FFT.
 *
 * Parity: every function here is pinned by tests against closed forms,
 * library special functions or invariants (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* HEALPix ring geometry.  Rings are numbered i = 1 .. 4n-1 from north to      */
/* south.  North cap i < n: z = 1 - i^2/(3n^2), 4i pixels at                   */
/* phi = (k + 1/2) pi/(2i).  Belt n <= i <= 3n: z = 4/3 - 2i/(3n), 4n pixels    */
/* at phi = (k + f/2) pi/(2n), f = 1 when i - n is even else 0 (the standard    */
/* RING numbering, first pixel at phi = 0 on the shifted rings).  South cap is  */
/* the mirror image of the north cap.                                            */
/* ------------------------------------------------------------------------- */
static void ring_geom(int64_t n, int64_t i, double *z, double *sth,
                      int64_t *len, int64_t *start, double *phi0)
{
    double omz, opz; /* 1 - z and 1 + z, kept separately near the poles */
    if (i < n) {
        omz = (double)(i * i) / (3.0 * (double)(n * n));
        *z = 1.0 - omz;
        opz = 2.0 - omz;
        *len = 4 * i;
        *start = 2 * i * (i - 1);
        *phi0 = M_PI / (4.0 * (double)i);
    } else if (i <= 3 * n) {
        *z = (double)(4 * n - 2 * i) / (3.0 * (double)n);
        omz = 1.0 - *z;
        opz = 1.0 + *z;
        *len = 4 * n;
        *start = 2 * n * (n - 1) + 4 * n * (i - n);
        *phi0 = (((i - n) % 2) == 0) ? M_PI / (4.0 * (double)n) : 0.0;
    } else {
        int64_t ip = 4 * n - i;
        opz = (double)(ip * ip) / (3.0 * (double)(n * n));
        *z = opz - 1.0;
        omz = 2.0 - opz;
        *len = 4 * ip;
        *start = 12 * n * n - 2 * ip * (ip + 1);
        *phi0 = M_PI / (4.0 * (double)ip);
    }
    *sth = sqrt(omz * opz);
}

/* Ring table for nside n: arrays of length 4n-1. */
int orc_ring_table(int64_t n, double *z, double *sth, int64_t *len,
                   int64_t *start, double *phi0)
{
    if (n < 1) return -1;
    for (int64_t i = 1; i <= 4 * n - 1; ++i)
        ring_geom(n, i, &z[i - 1], &sth[i - 1], &len[i - 1], &start[i - 1],
                  &phi0[i - 1]);
    return 0;
}

/* Unit vectors of all 12 n^2 pixel centres, RING order, xyz interleaved. */
int orc_pix2vec(int64_t n, double *xyz)
{
    if (n < 1) return -1;
    for (int64_t i = 1; i <= 4 * n - 1; ++i) {
        double z, s, phi0;
        int64_t len, start;
        ring_geom(n, i, &z, &s, &len, &start, &phi0);
        double dphi = 2.0 * M_PI / (double)len;
        for (int64_t k = 0; k < len; ++k) {
            double phi = phi0 + dphi * (double)k;
            double *r = xyz + 3 * (start + k);
            r[0] = s * cos(phi);
            r[1] = s * sin(phi);
            r[2] = z;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Legendre sums (Eq. 1's operator P_{l theta}, applied in the inverse        */
/* direction): K(z) = sum_{l=0}^{lmax} (2l+1)/(4 pi) c_l P_l(z) and its z-      */
/* derivative, by the three-term recurrence                                      */
/*   (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1},                                   */
/*   P'_{l+1} = P'_{l-1} + (2l+1) P_l.                                           */
/* ------------------------------------------------------------------------- */
static void legendre_sum1(int lmax, const double *c, double z, double *K,
                          double *dK)
{
    double p0 = 1.0, p1 = z;     /* P_{l}, P_{l+1} */
    double d0 = 0.0, d1 = 1.0;   /* P'_{l}, P'_{l+1} */
    double sk = c[0] * 1.0 / (4.0 * M_PI);
    double sd = 0.0;
    if (lmax >= 1) {
        sk += c[1] * 3.0 / (4.0 * M_PI) * p1;
        sd += c[1] * 3.0 / (4.0 * M_PI) * d1;
    }
    for (int l = 1; l < lmax; ++l) {
        double p2 = ((2.0 * l + 1.0) * z * p1 - (double)l * p0) / (double)(l + 1);
        double d2 = d0 + (2.0 * l + 1.0) * p1;
        double f = (2.0 * (l + 1) + 1.0) / (4.0 * M_PI) * c[l + 1];
        sk += f * p2;
        sd += f * d2;
        p0 = p1; p1 = p2;
        d0 = d1; d1 = d2;
    }
    *K = sk;
    if (dK) *dK = sd;
}

int orc_legendre_sum(int lmax, const double *c, int64_t npts, const double *z,
                     double *K, double *dK)
{
    if (lmax < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p)
        legendre_sum1(lmax, c, z[p], &K[p], dK ? &dK[p] : NULL);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Brute-force real-space convolution.                                         */
/*                                                                             */
/*   out_i = (4 pi / Npix) sum_{all j, theta_ij <= theta_cut} K(theta_ij) m_j   */
/*                                                                             */
/* theta <= theta_cut is tested as chord^2 <= (2 sin(theta_cut/2))^2 with the   */
/* chord |r_i - r_j| from FP64 unit vectors.  Kernel modes:                      */
/*   kmode 0: K from the Legendre sum of c[0..lmax] at z = 1 - chord^2/2        */
/*            (the exact truncated kernel);                                      */
/*   kmode 1: K from a cubic Hermite interpolant in the chord d on n_int equal  */
/*            intervals of [0, d_cut], node values tabK[k] and node             */
/*            derivatives tabD[k] = dK/dd (the tabulated kernel).               */
/* ambig[i] (optional) receives sum |K m| dOmega over pairs whose chord^2 lies  */
/* within amb_eps * d_cut^2 of the cut, i.e. pairs whose inclusion a            */
/* reduced-precision implementation may legitimately decide the other way.     */
/* ------------------------------------------------------------------------- */
static double hermite_eval(int64_t n_int, double h, const double *tabK,
                           const double *tabD, double d)
{
    double u = d / h;
    int64_t k = (int64_t)floor(u);
    if (k < 0) k = 0;
    if (k > n_int - 1) k = n_int - 1;
    double t = u - (double)k;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    return h00 * tabK[k] + h10 * h * tabD[k] + h01 * tabK[k + 1] +
           h11 * h * tabD[k + 1];
}

int orc_brute_conv(int64_t nside, const double *map, int64_t n_out,
                   const int64_t *out_pix, int kmode, int lmax, const double *c,
                   int64_t n_int, const double *tabK, const double *tabD,
                   double theta_cut, double amb_eps, double *out, double *ambig)
{
    if (nside < 1 || n_out < 0) return -1;
    if (kmode == 0 && (lmax < 0 || !c)) return -1;
    if (kmode == 1 && (n_int < 1 || !tabK || !tabD)) return -1;
    int64_t npix = 12 * nside * nside;
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)npix);
    if (!xyz) return -2;
    orc_pix2vec(nside, xyz);
    double dcut = 2.0 * sin(0.5 * theta_cut);
    double dcut2 = dcut * dcut;
    double h = dcut / (double)(n_int > 0 ? n_int : 1);
    /* theta_cut >= pi: the whole sphere, antipodal pairs included whatever the
       rounding of their chord */
    if (theta_cut >= M_PI) dcut2 = HUGE_VAL;
    double domega = 4.0 * M_PI / (double)npix;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = out_pix ? out_pix[o] : o;
        const double *ri = xyz + 3 * i;
        double acc = 0.0, amb = 0.0;
        for (int64_t j = 0; j < npix; ++j) {
            const double *rj = xyz + 3 * j;
            double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 > dcut2 * (1.0 + amb_eps)) continue; /* outside the cap */
            double kv;
            if (kmode == 0) {
                legendre_sum1(lmax, c, 1.0 - 0.5 * d2, &kv, NULL);
            } else {
                double d = sqrt(d2);
                if (d > dcut) d = dcut;
                kv = hermite_eval(n_int, h, tabK, tabD, d);
            }
            double term = kv * map[j] * domega;
            if (dcut2 < HUGE_VAL && fabs(d2 - dcut2) <= amb_eps * dcut2)
                amb += fabs(term);
            if (d2 <= dcut2) acc += term;
        }
        out[o] = acc;
        if (ambig) ambig[o] = amb;
    }
    free(xyz);
    return 0;
}

/* Number of ordered pixel pairs (i, j) with theta_ij <= theta_cut, for the    */
/* output pixels listed (all pixels when out_pix is NULL).                     */
int orc_count_pairs(int64_t nside, int64_t n_out, const int64_t *out_pix,
                    double theta_cut, int64_t *counts)
{
    int64_t npix = 12 * nside * nside;
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)npix);
    if (!xyz) return -2;
    orc_pix2vec(nside, xyz);
    double dcut = 2.0 * sin(0.5 * theta_cut);
    double dcut2 = dcut * dcut;
    if (theta_cut >= M_PI) dcut2 = HUGE_VAL;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t o = 0; o < n_out; ++o) {
        int64_t i = out_pix ? out_pix[o] : o;
        const double *ri = xyz + 3 * i;
        int64_t cnt = 0;
        for (int64_t j = 0; j < npix; ++j) {
            const double *rj = xyz + 3 * j;
            double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
            if (dx * dx + dy * dy + dz * dz <= dcut2) ++cnt;
        }
        counts[o] = cnt;
    }
    free(xyz);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Normalised associated Legendre functions lambda_lm(z), with                 */
/* Y_lm(theta, phi) = lambda_lm(cos theta) e^{i m phi} orthonormal on the       */
/* sphere (no Condon-Shortley phase).  Recurrences:                             */
/*   lambda_mm = sqrt((2m+1)/(4 pi) prod_{k=1}^m (2k-1)/(2k)) sin^m theta       */
/*   lambda_{m+1,m} = z sqrt(2m+3) lambda_mm                                    */
/*   lambda_lm = a_lm z lambda_{l-1,m} - b_lm lambda_{l-2,m},                   */
/*   a_lm = sqrt((4l^2-1)/(l^2-m^2)),                                            */
/*   b_lm = sqrt((2l+1)((l-1)^2-m^2) / ((2l-3)(l^2-m^2))).                      */
/* lambda_mm underflows double precision for large m away from the equator,    */
/* so values are carried as v * BIG^e with an integer exponent e.              */
/* ------------------------------------------------------------------------- */
#define ORC_LOGBIG (200.0 * 0.69314718055994530942)
#define ORC_BIG 1.6069380442589903e+60 /* 2^200 */

/* Fill lam[l - m] = lambda_lm(z) for l = m .. lmax. */
static void lambda_column(int lmax, int m, double z, double sth,
                          const double *a, const double *b, double logfac_m,
                          double *lam)
{
    if (sth <= 0.0) {
        for (int l = m; l <= lmax; ++l)
            lam[l - m] = 0.0;
        if (m == 0)
            for (int l = 0; l <= lmax; ++l)
                lam[l] = sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) *
                         ((z < 0.0 && (l % 2)) ? -1.0 : 1.0);
        return;
    }
    double loglam = logfac_m + (double)m * log(sth);
    int e = (int)floor(loglam / ORC_LOGBIG);
    double v0 = exp(loglam - (double)e * ORC_LOGBIG);
    double vprev = 0.0, vcur = v0;
    for (int l = m; l <= lmax; ++l) {
        if (l > m) {
            double vn;
            if (l == m + 1)
                vn = z * sqrt(2.0 * m + 3.0) * vcur;
            else
                vn = a[l] * z * vcur - b[l] * vprev;
            vprev = vcur;
            vcur = vn;
            if (fabs(vcur) > ORC_BIG) {
                vcur /= ORC_BIG;
                vprev /= ORC_BIG;
                e += 1;
            }
        }
        double val;
        if (e == 0) val = vcur;
        else if (e < -4) val = 0.0;
        else val = ldexp(vcur, 200 * e);
        lam[l - m] = val;
    }
}

static void recurrence_coeffs(int lmax, int m, double *a, double *b)
{
    for (int l = m + 2; l <= lmax; ++l) {
        double l2 = (double)l * l, m2 = (double)m * m;
        a[l] = sqrt((4.0 * l2 - 1.0) / (l2 - m2));
        b[l] = sqrt((2.0 * l + 1.0) * ((l - 1.0) * (l - 1.0) - m2) /
                    ((2.0 * l - 3.0) * (l2 - m2)));
    }
}

static double log_lambda_mm_factor(int m)
{
    double s = 0.0;
    for (int k = 1; k <= m; ++k)
        s += log((2.0 * k - 1.0) / (2.0 * k));
    return 0.5 * (log((2.0 * m + 1.0) / (4.0 * M_PI)) + s);
}

/* lambda_lm(z) for all l <= lmax, m <= min(l, mmax) at the given points;     */
/* output layout [p][alm_index(l, m)] with alm_index(l,m) = m(2 lmax+1-m)/2+l. */
int orc_lambda_table(int lmax, int mmax, int64_t npts, const double *z,
                     double *out)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax) return -1;
    int64_t nalm = (int64_t)(mmax + 1) * (2 * lmax + 2 - mmax) / 2;
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * (lmax + 2));
        double *b = (double *)malloc(sizeof(double) * (lmax + 2));
        double *lam = (double *)malloc(sizeof(double) * (lmax + 2));
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= mmax; ++m) {
            recurrence_coeffs(lmax, m, a, b);
            double lf = log_lambda_mm_factor(m);
            int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
            for (int64_t p = 0; p < npts; ++p) {
                double zz = z[p];
                double s = sqrt((1.0 - zz) * (1.0 + zz));
                lambda_column(lmax, m, zz, s, a, b, lf, lam);
                for (int l = m; l <= lmax; ++l)
                    out[p * nalm + base + l] = lam[l - m];
            }
        }
        free(a); free(b); free(lam);
    }
    (void)nalm;
    return 0;
}

/* Legendre stage of the analysis: alm[idx(l,m)] = w * sum_r lambda_lm(z_r)    */
/* F[r][m], with F[r][m] = sum_k map_{r,k} e^{-i m phi_{r,k}} (the ring sums)   */
/* and w = 4 pi / Npix the equal-area quadrature weight.                        */
int orc_alm_analysis(int lmax, int mmax, int64_t nrings, const double *z,
                     const double *sth, const double complex *F, double w,
                     double complex *alm)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax) return -1;
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * (lmax + 2));
        double *b = (double *)malloc(sizeof(double) * (lmax + 2));
        double *lam = (double *)malloc(sizeof(double) * (lmax + 2));
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= mmax; ++m) {
            recurrence_coeffs(lmax, m, a, b);
            double lf = log_lambda_mm_factor(m);
            int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
            for (int l = m; l <= lmax; ++l) alm[base + l] = 0.0;
            for (int64_t r = 0; r < nrings; ++r) {
                lambda_column(lmax, m, z[r], sth[r], a, b, lf, lam);
                double complex f = F[r * (mmax + 1) + m] * w;
                for (int l = m; l <= lmax; ++l)
                    alm[base + l] += lam[l - m] * f;
            }
        }
        free(a); free(b); free(lam);
    }
    return 0;
}

/* Legendre stage of the synthesis: G[r][m] = sum_l alm[idx(l,m)] lambda_lm(z_r). */
int orc_alm_synthesis(int lmax, int mmax, int64_t nrings, const double *z,
                      const double *sth, const double complex *alm,
                      double complex *G)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax) return -1;
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * (lmax + 2));
        double *b = (double *)malloc(sizeof(double) * (lmax + 2));
        double *lam = (double *)malloc(sizeof(double) * (lmax + 2));
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m <= mmax; ++m) {
            recurrence_coeffs(lmax, m, a, b);
            double lf = log_lambda_mm_factor(m);
            int64_t base = (int64_t)m * (2 * lmax + 1 - m) / 2;
            for (int64_t r = 0; r < nrings; ++r) {
                lambda_column(lmax, m, z[r], sth[r], a, b, lf, lam);
                double complex g = 0.0;
                for (int l = m; l <= lmax; ++l)
                    g += alm[base + l] * lam[l - m];
                G[r * (mmax + 1) + m] = g;
            }
        }
        free(a); free(b); free(lam);
    }
    return 0;
}
