// Host FP64 kernel split: the weighted least-squares fit of Sec. 2, Eq. 1-6.
//
// Unknowns (Eq. 4): Khat_l for l <= l_cut and z_cut real-space coefficients x_j
// attached to the Gauss-Legendre nodes z_j (of an oversample*(lmax+1)-point
// rule) inside the cap z >= cos(theta_cut).  Real-space basis function j is
// the band-limited projection f_j(z) = w_j sum_l (2l+1)/2 P_l(z_j) P_l(z),
// truncated at theta_cut; column j of the Legendre operator P (Eq. 1, Eq. 5) is
// its exact transform A_{lj} = 2 pi int_{cos theta_cut}^1 f_j P_l dz, evaluated
// with an (lmax+1)-point Gauss rule on [cos theta_cut, 1].
//
// Solve (Eq. 3): every row l <= l_cut has its own free unknown Khat_l, so those
// rows are fitted exactly (Khat_l = K_l - (A x)_l) and the minimisation of
// Eq. 2 reduces to the rows l > l_cut.  That block, W^{1/2} A with unit-norm
// columns, is solved by SVD (Householder QR, then one-sided Jacobi on R).  The
// cut of Sec. 2 (1e-6) is on the singular values of the normal matrix of
// Eq. 3, i.e. W^{1/2} A's singular values below sqrt(rcond) * max are dropped.
//
// The resulting real-space kernel is K_r(z) = sum_l (2l+1)/(4 pi) c_l P_l(z)
// for z >= cos(theta_cut), c_l = 2 pi sum_j w_j x_j P_l(z_j), zero outside.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ksc_internal.h"

namespace ksc {
namespace {

constexpr double kPi = 3.14159265358979323846;

// P_n(x) and P_{n-1}(x) by the three-term recurrence.
void legendre_pair(int n, double x, double *pn, double *pnm1) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *pnm1 = 0.0; return; }
    for (int l = 1; l < n; ++l) {
        double p2 = ((2.0 * l + 1.0) * x * p1 - l * p0) / (l + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pnm1 = p0;
}

// i-th (1-based, descending) node and weight of the n-point Gauss-Legendre rule
// on [-1, 1], by Newton's method from the asymptotic guess.
void gauss_node(int n, int i, double *x, double *w) {
    double z = std::cos(kPi * (i - 0.25) / (n + 0.5));
    double pn, pm;
    for (int it = 0; it < 100; ++it) {
        legendre_pair(n, z, &pn, &pm);
        double dp = n * (z * pn - pm) / (z * z - 1.0);
        double dz = pn / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
    }
    legendre_pair(n, z, &pn, &pm);
    double dp = n * (z * pn - pm) / (z * z - 1.0);
    *x = z;
    *w = 2.0 / ((1.0 - z * z) * dp * dp);
}

// P_l(x), l = 0..lmax, into row[0..lmax].
void legendre_row(int lmax, double x, double *row) {
    row[0] = 1.0;
    if (lmax >= 1) row[1] = x;
    for (int l = 1; l < lmax; ++l)
        row[l + 1] = ((2.0 * l + 1.0) * x * row[l] - l * row[l - 1]) / (l + 1.0);
}

// One-sided Jacobi SVD of the column-major p x n matrix R (columns are
// orthogonalised in place; V accumulates the rotations, n x n column-major).
bool jacobi_svd(int p, int n, std::vector<double> &R, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) V[(size_t)j * n + j] = 1.0;
    // columns whose squared norm is below tiny * ||R||_F^2 are numerically null:
    // rotating them against each other only shuffles rounding noise
    double fro = 0.0;
    for (size_t k = 0; k < (size_t)p * n; ++k) fro += R[k] * R[k];
    const double tiny = 1e-28 * fro;
    for (int sweep = 0; sweep < 200; ++sweep) {
        bool rotated = false;
        for (int a = 0; a < n - 1; ++a) {
            double *ca = &R[(size_t)a * p];
            for (int b = a + 1; b < n; ++b) {
                double *cb = &R[(size_t)b * p];
                double al = 0, be = 0, ga = 0;
                for (int k = 0; k < p; ++k) {
                    al += ca[k] * ca[k];
                    be += cb[k] * cb[k];
                    ga += ca[k] * cb[k];
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-15 * std::sqrt(al * be)) continue;
                if (al < tiny || be < tiny) continue;
                rotated = true;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) /
                           (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int k = 0; k < p; ++k) {
                    double u = ca[k], v = cb[k];
                    ca[k] = c * u - s * v;
                    cb[k] = s * u + c * v;
                }
                double *va = &V[(size_t)a * n], *vb = &V[(size_t)b * n];
                for (int k = 0; k < n; ++k) {
                    double u = va[k], v = vb[k];
                    va[k] = c * u - s * v;
                    vb[k] = s * u + c * v;
                }
            }
        }
        if (!rotated) return true;
    }
    return false;
}

} // namespace

double sigma_rms_eq2(const double *K, const double *Kt, const double *cl, int lmax) {
    double s = 0.0;
    for (int l = 0; l <= lmax; ++l) {
        double d = K[l] - Kt[l];
        s += d * d * (cl ? cl[l] : 1.0) * (2.0 * l + 1.0);
    }
    return std::sqrt(s / (4.0 * kPi));
}

double frac_error_eq6(const double *K, const double *Kt, const double *cl, int lmax,
                      double alpha) {
    double den = 0.0;
    for (int l = 0; l <= lmax; ++l) den += (2.0 * l + 1.0) * K[l] * K[l] * (cl ? cl[l] : 1.0);
    den /= 4.0 * kPi;
    if (den <= 0.0) return 0.0;
    return alpha * sigma_rms_eq2(K, Kt, cl, lmax) / std::sqrt(den);
}

int fit_split_lsq(const double *K, int lmax, int l_cut, double theta_cut,
                  const double *cl_in, int oversample, double rcond, int n_constraints,
                  FitResult *out, std::string *msg) {
    const int L = lmax + 1;
    const double zc = std::cos(theta_cut);

    // Real-space nodes: the Gauss-Legendre nodes inside the cap.
    const int nbig = oversample * L;
    std::vector<double> zj, wj;
    for (int i = 1; i <= nbig; ++i) {
        double x, w;
        gauss_node(nbig, i, &x, &w);
        if (x < zc) break;
        zj.push_back(x);
        wj.push_back(w);
    }
    const int nz = (int)zj.size();
    if (nz == 0) {
        *msg = "theta_cut is below the node spacing of the real-space basis";
        return KSC_ERR_ARG;
    }

    // Gauss rule on [zc, 1] with L points (exact for the degree-2 lmax integrand).
    const int nq = L;
    std::vector<double> zq(nq), wq(nq);
    for (int i = 1; i <= (nq + 1) / 2; ++i) {
        double x, w;
        gauss_node(nq, i, &x, &w);
        zq[i - 1] = x;
        wq[i - 1] = w;
        zq[nq - i] = -x;
        wq[nq - i] = w;
    }
    for (int q = 0; q < nq; ++q) {
        zq[q] = zc + (zq[q] + 1.0) * (1.0 - zc) / 2.0;
        wq[q] *= (1.0 - zc) / 2.0;
    }

    // Legendre rows at the nodes.
    std::vector<double> Pj((size_t)nz * L), Pq((size_t)nq * L);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < nz; ++j) legendre_row(lmax, zj[j], &Pj[(size_t)j * L]);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < nq; ++q) legendre_row(lmax, zq[q], &Pq[(size_t)q * L]);

    // G[l][j] = (2l+1)/2 w_j P_l(z_j)
    std::vector<double> G((size_t)L * nz);
    for (int l = 0; l < L; ++l)
        for (int j = 0; j < nz; ++j)
            G[(size_t)l * nz + j] = 0.5 * (2.0 * l + 1.0) * wj[j] * Pj[(size_t)j * L + l];

    // F[q][j] = f_j(zq_q) = sum_l P_l(zq_q) G[l][j]
    std::vector<double> F((size_t)nq * nz, 0.0);
#pragma omp parallel for schedule(dynamic, 8)
    for (int q = 0; q < nq; ++q) {
        double *f = &F[(size_t)q * nz];
        const double *pr = &Pq[(size_t)q * L];
        for (int l = 0; l < L; ++l) {
            double a = pr[l];
            const double *g = &G[(size_t)l * nz];
            for (int j = 0; j < nz; ++j) f[j] += a * g[j];
        }
        for (int j = 0; j < nz; ++j) f[j] *= wq[q];
    }

    // A[l][j] = 2 pi sum_q wq_q P_l(zq_q) f_j(zq_q)
    std::vector<double> A((size_t)L * nz, 0.0);
    const int LB = 32;
#pragma omp parallel for schedule(dynamic, 1)
    for (int lb = 0; lb < L; lb += LB) {
        int le = std::min(L, lb + LB);
        for (int q = 0; q < nq; ++q) {
            const double *pr = &Pq[(size_t)q * L];
            const double *f = &F[(size_t)q * nz];
            for (int l = lb; l < le; ++l) {
                double a = pr[l];
                double *row = &A[(size_t)l * nz];
                for (int j = 0; j < nz; ++j) row[j] += a * f[j];
            }
        }
        for (int l = lb; l < le; ++l)
            for (int j = 0; j < nz; ++j) A[(size_t)l * nz + j] *= 2.0 * kPi;
    }
    std::vector<double>().swap(Pq);
    std::vector<double>().swap(F);

    // Continuity at the cut (reading of Sec. 2's truncation "to a limit
    // theta_cut"): the real-space kernel K_r = sum_j x_j f_j is made to vanish
    // at z_cut (n_constraints >= 1) with zero slope there (2) by eliminating the
    // unknowns at the nodes nearest the cut (the last ones, nodes descend to
    // z_cut): C_E x_E + C_F x_F = 0 with rows f_j(z_cut), f_j'(z_cut).  A jump
    // at the cut would make the pixel sum over-/under-count boundary pixels.
    const int nc = std::min(std::max(n_constraints, 0), std::max(nz - 1, 0));
    const int nf = nz - nc;
    // x = T t: T is nz x nf, identity on the free nodes 0..nf-1
    std::vector<double> TE((size_t)nc * nf, 0.0);  // rows of T for the eliminated nodes
    if (nc > 0) {
        std::vector<double> pc(L), dc(L);
        pc[0] = 1.0; dc[0] = 0.0;
        if (lmax >= 1) { pc[1] = zc; dc[1] = 1.0; }
        for (int l = 1; l < lmax; ++l) {
            pc[l + 1] = ((2.0 * l + 1.0) * zc * pc[l] - (double)l * pc[l - 1]) / (double)(l + 1);
            dc[l + 1] = dc[l - 1] + (2.0 * l + 1.0) * pc[l];
        }
        std::vector<double> cg(nz, 0.0), ch(nz, 0.0);  // f_j(z_cut), f_j'(z_cut)
        for (int l = 0; l < L; ++l)
            for (int j = 0; j < nz; ++j) {
                cg[j] += G[(size_t)l * nz + j] * pc[l];
                ch[j] += G[(size_t)l * nz + j] * dc[l];
            }
        if (nc == 1) {
            const double ge = cg[nz - 1];
            if (!(std::fabs(ge) > 0.0)) {
                *msg = "continuity constraint is singular at this theta_cut";
                return KSC_ERR_SVD;
            }
            for (int f = 0; f < nf; ++f) TE[f] = -cg[f] / ge;
        } else {
            // [g_a g_b; h_a h_b] x_E = -[g_F; h_F] x_F, a = nz-2, b = nz-1
            const double a11 = cg[nz - 2], a12 = cg[nz - 1], a21 = ch[nz - 2], a22 = ch[nz - 1];
            const double det = a11 * a22 - a12 * a21;
            const double scale = std::fabs(a11 * a22) + std::fabs(a12 * a21);
            if (!(std::fabs(det) > 1e-12 * scale)) {
                *msg = "continuity constraint is singular at this theta_cut";
                return KSC_ERR_SVD;
            }
            for (int f = 0; f < nf; ++f) {
                const double rg = -cg[f], rh = -ch[f];
                TE[f] = (rg * a22 - a12 * rh) / det;
                TE[(size_t)nf + f] = (a11 * rh - a21 * rg) / det;
            }
        }
    }
    // Columns of the constrained operator: A T (L x nf)
    std::vector<double> AT((size_t)L * nf);
    for (int l = 0; l < L; ++l) {
        const double *row = &A[(size_t)l * nz];
        double *o = &AT[(size_t)l * nf];
        for (int f = 0; f < nf; ++f) {
            double v = row[f];
            for (int e = 0; e < nc; ++e) v += row[nf + e] * TE[(size_t)e * nf + f];
            o[f] = v;
        }
    }

    // Reduced weighted system on rows l > l_cut, unit-norm columns.
    const int m = lmax - l_cut;
    std::vector<double> Bm((size_t)nf * m);  // column-major m x nf
    std::vector<double> bv(m), cn(nf, 0.0);
    for (int i = 0; i < m; ++i) {
        int l = l_cut + 1 + i;
        double sw = std::sqrt((2.0 * l + 1.0) * (cl_in ? cl_in[l] : 1.0));
        bv[i] = sw * K[l];
        for (int j = 0; j < nf; ++j) Bm[(size_t)j * m + i] = sw * AT[(size_t)l * nf + j];
    }
    std::vector<double>().swap(AT);
    for (int j = 0; j < nf; ++j) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += Bm[(size_t)j * m + i] * Bm[(size_t)j * m + i];
        cn[j] = s > 0 ? std::sqrt(s) : 1.0;
        for (int i = 0; i < m; ++i) Bm[(size_t)j * m + i] /= cn[j];
    }

    // Householder QR when tall: R (p x nf, column-major), c = Q^T b.
    int p = m;
    std::vector<double> R, cvec;
    if (m > nf) {
        for (int j = 0; j < nf; ++j) {
            double *col = &Bm[(size_t)j * m];
            double nrm = 0;
            for (int i = j; i < m; ++i) nrm += col[i] * col[i];
            nrm = std::sqrt(nrm);
            if (nrm == 0.0) continue;
            double alpha = col[j] > 0 ? -nrm : nrm;
            std::vector<double> v(col + j, col + m);
            v[0] -= alpha;
            double vn = 0;
            for (double e : v) vn += e * e;
            if (vn == 0.0) continue;
            for (int jj = j; jj < nf; ++jj) {
                double *cc = &Bm[(size_t)jj * m];
                double d = 0;
                for (int i = j; i < m; ++i) d += v[i - j] * cc[i];
                d = 2.0 * d / vn;
                for (int i = j; i < m; ++i) cc[i] -= d * v[i - j];
            }
            double d = 0;
            for (int i = j; i < m; ++i) d += v[i - j] * bv[i];
            d = 2.0 * d / vn;
            for (int i = j; i < m; ++i) bv[i] -= d * v[i - j];
        }
        p = nf;
        R.assign((size_t)nf * nf, 0.0);
        for (int j = 0; j < nf; ++j)
            for (int i = 0; i <= j; ++i) R[(size_t)j * nf + i] = Bm[(size_t)j * m + i];
        cvec.assign(bv.begin(), bv.begin() + nf);
    } else {
        R = Bm;
        cvec = bv;
    }
    std::vector<double>().swap(Bm);

    std::vector<double> V;
    if (!jacobi_svd(p, nf, R, V)) {
        *msg = "one-sided Jacobi SVD did not converge";
        return KSC_ERR_SVD;
    }
    std::vector<double> sig(nf);
    double smax = 0;
    for (int j = 0; j < nf; ++j) {
        double s = 0;
        for (int k = 0; k < p; ++k) s += R[(size_t)j * p + k] * R[(size_t)j * p + k];
        sig[j] = std::sqrt(s);
        smax = std::max(smax, sig[j]);
    }
    // The cut of Sec. 2 applies to the singular values of the normal matrix
    // A^T W A (Eq. 3), the squares of those of W^{1/2} A.
    const double cut = std::sqrt(rcond) * smax;
    std::vector<double> y(nf, 0.0);
    int kept = 0;
    for (int j = 0; j < nf; ++j) {
        if (!(sig[j] > cut)) continue;
        ++kept;
        double d = 0;
        for (int k = 0; k < p; ++k) d += R[(size_t)j * p + k] * cvec[k];
        d /= sig[j] * sig[j];  // (u_j . c) / sigma_j with u_j = R_j / sigma_j
        for (int k = 0; k < nf; ++k) y[k] += V[(size_t)j * nf + k] * d;
    }
    std::vector<double> x(nz);
    for (int j = 0; j < nf; ++j) x[j] = y[j] / cn[j];
    for (int e = 0; e < nc; ++e) {
        double v = 0.0;
        for (int f = 0; f < nf; ++f) v += TE[(size_t)e * nf + f] * x[f];
        x[nf + e] = v;
    }

    // Outputs: K~ (Eq. 1), Khat_l, c_real.
    out->k_tilde.assign(L, 0.0);
    out->k_harm.assign(l_cut + 1, 0.0);
    for (int l = 0; l < L; ++l) {
        double ax = 0;
        for (int j = 0; j < nz; ++j) ax += A[(size_t)l * nz + j] * x[j];
        if (l <= l_cut) {
            out->k_harm[l] = K[l] - ax;
            out->k_tilde[l] = K[l];
        } else {
            out->k_tilde[l] = ax;
        }
    }
    out->c_real.assign(L, 0.0);
    for (int j = 0; j < nz; ++j) {
        double f = 2.0 * kPi * wj[j] * x[j];
        const double *pr = &Pj[(size_t)j * L];
        for (int l = 0; l < L; ++l) out->c_real[l] += f * pr[l];
    }
    out->n_unknowns = nf;
    out->n_kept = kept;
    return KSC_OK;
}

// ---------------------------------------------------------------------------
// HEALPix RING geometry (Gorski et al. 2005).
// ---------------------------------------------------------------------------
void ring_geometry(int n, RingGeom *g) {
    const int nr = 4 * n - 1;
    g->z.resize(nr); g->s.resize(nr);
    g->len.resize(nr); g->start.resize(nr); g->phase.resize(nr);
    const double nn = (double)n;
    for (int r = 0; r < nr; ++r) {
        const long long i = r + 1;
        double z, omz, opz;
        if (i < n) {                       // north polar cap
            omz = (double)(i * i) / (3.0 * nn * nn);
            z = 1.0 - omz; opz = 1.0 + z;
            g->len[r] = (int)(4 * i);
            g->start[r] = (int)(2 * i * (i - 1));
            g->phase[r] = 1;
        } else if (i <= 3LL * n) {         // equatorial belt
            z = (double)(4LL * n - 2 * i) / (3.0 * nn);
            omz = 1.0 - z; opz = 1.0 + z;
            g->len[r] = 4 * n;
            g->start[r] = (int)(2LL * n * (n - 1) + 4LL * n * (i - n));
            g->phase[r] = ((i - n) % 2 == 0) ? 1 : 0;
        } else {                           // south polar cap (mirror)
            const long long ip = 4LL * n - i;
            opz = (double)(ip * ip) / (3.0 * nn * nn);
            z = opz - 1.0; omz = 1.0 - z;
            g->len[r] = (int)(4 * ip);
            g->start[r] = (int)(12LL * n * n - 2 * ip * (ip + 1));
            g->phase[r] = 1;
        }
        g->z[r] = z;
        g->s[r] = std::sqrt(omz * opz);
    }
}

} // namespace ksc
