// Split planning on the host (declared in include/ksconv.h): the cost models of
// the two halves of the split convolution (Sec. 2, Eq. 7-8 refitted for this
// library), the surrogate's input features, and the scanning strategy of Sec. 2
// that picks the cheapest (l_cut, theta_cut) meeting an error bound.
//
// Cost models.  The GPU half (the real-space sum) costs a fixed amount per
// in-disc pixel pair plus a per-ring-pair overhead (table build, staging) that,
// at a given pair count, grows as the rings shorten: t_gpu = g0 + (g1 + g2 1000 /
// nside) P(nside, theta_cut), with P the pair count of a disc of radius theta_cut
// on a map of Npix pixels, P = Npix^2 (1 - cos theta_cut) / 2 (the paper's Eq. 7
// is linear in theta_cut for its GTX 480 code).  The host half (an
// SHT to l_cut on a map with l_max) follows Eq. 8, t_host = h0 + h1 l_cut^2 l_max
// / 4096^3 (the paper's h1 = 160 s for one 2.8 GHz core).  Both are fitted by
// least squares in relative error to measured times.
//
// Scan (Sec. 2): a linear scan over theta_cut on a grid; for each theta_cut a
// binary search for the smallest l_cut whose fitted split meets the Eq. 6 bound
// (the error is taken as falling with l_cut, as Sec. 2 does; where it does not,
// the search returns one l_cut meeting the bound), or, as an option, an ascending
// pass over evenly spaced l_cut followed by bisection inside the first step that
// meets the bound; the candidate of least max(t_gpu, t_host) wins -- the two
// halves run concurrently (Fig. 1).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ksc_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kArcmin = kPi / (180.0 * 60.0);

int sfail(int code, const std::string &msg) {
    ksc::set_last_error(msg);
    return code;
}

// Least squares of t_i ~ sum_j c_j X_ij in relative error -- minimise
// sum_i ((X c)_i / t_i - 1)^2 -- with every c_j >= 0: the unconstrained solve on each
// subset of the columns (normal equations, Gaussian elimination with partial
// pivoting; at most three columns), the feasible solution of least residual.
bool fit_rel(const std::vector<std::vector<double>> &X, const std::vector<double> &t,
             std::vector<double> *c) {
    const int k = (int)X.size();
    double best = INFINITY;
    std::vector<double> keep(k, 0.0);
    for (int mask = 1; mask < (1 << k); ++mask) {
        std::vector<int> col;
        for (int j = 0; j < k; ++j)
            if (mask >> j & 1) col.push_back(j);
        const int m = (int)col.size();
        std::vector<double> A(m * (m + 1), 0.0);  // [N | r], N = B^T B, r = B^T 1
        for (size_t i = 0; i < t.size(); ++i)
            for (int a = 0; a < m; ++a) {
                const double u = X[col[a]][i] / t[i];
                A[a * (m + 1) + m] += u;
                for (int b2 = 0; b2 < m; ++b2) A[a * (m + 1) + b2] += u * X[col[b2]][i] / t[i];
            }
        bool ok = true;
        for (int p = 0; p < m && ok; ++p) {
            int piv = p;
            for (int r = p + 1; r < m; ++r)
                if (std::fabs(A[r * (m + 1) + p]) > std::fabs(A[piv * (m + 1) + p])) piv = r;
            if (!(std::fabs(A[piv * (m + 1) + p]) > 1e-300)) { ok = false; break; }
            for (int q = 0; q <= m; ++q) std::swap(A[p * (m + 1) + q], A[piv * (m + 1) + q]);
            for (int r = 0; r < m; ++r) {
                if (r == p) continue;
                const double f = A[r * (m + 1) + p] / A[p * (m + 1) + p];
                for (int q = p; q <= m; ++q) A[r * (m + 1) + q] -= f * A[p * (m + 1) + q];
            }
        }
        if (!ok) continue;
        std::vector<double> cc(k, 0.0);
        for (int a = 0; a < m; ++a) {
            cc[col[a]] = A[a * (m + 1) + m] / A[a * (m + 1) + a];
            if (!(cc[col[a]] >= 0.0) || !std::isfinite(cc[col[a]])) ok = false;
        }
        if (!ok) continue;
        double res = 0.0;
        for (size_t i = 0; i < t.size(); ++i) {
            double v = 0.0;
            for (int j = 0; j < k; ++j) v += cc[j] * X[j][i];
            res += (v / t[i] - 1.0) * (v / t[i] - 1.0);
        }
        if (res < best * (1.0 - 1e-12)) {
            best = res;
            keep = cc;
        }
    }
    if (!std::isfinite(best)) return false;
    *c = keep;
    return true;
}

double eq8_units(int l_cut, int lmax) {
    return (double)l_cut * (double)l_cut * (double)lmax / (4096.0 * 4096.0 * 4096.0);
}

} // namespace

extern "C" {

double ksc_cost_pairs(int nside, double theta_cut) {
    const double npix = 12.0 * (double)nside * (double)nside;
    const double th = std::min(std::max(theta_cut, 0.0), kPi);
    return npix * npix * 0.5 * (1.0 - std::cos(th));
}

int ksc_cost_model_default(ksc_cost_model *m) {
    if (!m) return sfail(KSC_ERR_ARG, "null model");
    // GPU: this library on one GB300 -- the nside-2048 benchmark (3.09e12 pairs,
    // 259 ms per map); host: Eq. 8 as printed (160 s on one 2.8 GHz core)
    m->gpu_ms0 = 0.1;
    m->gpu_ms_per_tpair = 259.0 / 3.085;
    m->gpu_ms_per_tpair_ring = 0.0;
    m->host_ms0 = 0.0;
    m->host_ms_eq8 = 160.0e3;
    return KSC_OK;
}

int ksc_cost_eval(const ksc_cost_model *m, int nside, int l_cut, int lmax, double theta_cut,
                  double *t_gpu_ms, double *t_host_ms) {
    if (!m) return sfail(KSC_ERR_ARG, "null model");
    if (nside < 1) return sfail(KSC_ERR_ARG, "nside < 1");
    if (t_gpu_ms)
        *t_gpu_ms = m->gpu_ms0 + (m->gpu_ms_per_tpair + m->gpu_ms_per_tpair_ring * 1000.0 / nside) *
                                     ksc_cost_pairs(nside, theta_cut) * 1e-12;
    if (t_host_ms)
        *t_host_ms = l_cut < 0 ? 0.0 : m->host_ms0 + m->host_ms_eq8 * eq8_units(l_cut, lmax);
    return KSC_OK;
}

int ksc_cost_fit_gpu(const int *nside, const double *theta_cut, const double *t_ms, int n,
                     ksc_cost_model *m) {
    if (!nside || !theta_cut || !t_ms || !m || n < 3) return sfail(KSC_ERR_ARG, "bad fit data");
    std::vector<std::vector<double>> X(3);
    std::vector<double> t;
    for (int i = 0; i < n; ++i) {
        if (!(t_ms[i] > 0.0) || nside[i] < 1) return sfail(KSC_ERR_ARG, "bad fit sample");
        const double p = ksc_cost_pairs(nside[i], theta_cut[i]) * 1e-12;
        X[0].push_back(1.0);
        X[1].push_back(p);
        X[2].push_back(p * 1000.0 / nside[i]);
        t.push_back(t_ms[i]);
    }
    bool one_nside = true;
    for (int i = 1; i < n; ++i) one_nside = one_nside && nside[i] == nside[0];
    if (one_nside) X.pop_back();  // the two pair terms coincide
    std::vector<double> c;
    if (!fit_rel(X, t, &c)) return sfail(KSC_ERR_ARG, "degenerate fit data");
    m->gpu_ms0 = c[0];
    m->gpu_ms_per_tpair = c[1];
    m->gpu_ms_per_tpair_ring = one_nside ? 0.0 : c[2];
    return KSC_OK;
}

int ksc_cost_fit_host(const int *l_cut, const int *lmax, const double *t_ms, int n,
                      ksc_cost_model *m) {
    if (!l_cut || !lmax || !t_ms || !m || n < 2) return sfail(KSC_ERR_ARG, "bad fit data");
    std::vector<std::vector<double>> X(2);
    std::vector<double> t;
    for (int i = 0; i < n; ++i) {
        if (!(t_ms[i] > 0.0) || l_cut[i] < 0 || lmax[i] < 1)
            return sfail(KSC_ERR_ARG, "bad fit sample");
        X[0].push_back(1.0);
        X[1].push_back(eq8_units(l_cut[i], lmax[i]));
        t.push_back(t_ms[i]);
    }
    std::vector<double> c;
    if (!fit_rel(X, t, &c)) return sfail(KSC_ERR_ARG, "degenerate fit data");
    m->host_ms0 = c[0];
    m->host_ms_eq8 = c[1];
    return KSC_OK;
}

int ksc_split_features(int n, const int *nside, const double *fwhm, const int *l_cut,
                       const double *theta_cut, float *x) {
    if (n < 0 || (n > 0 && (!nside || !fwhm || !l_cut || !theta_cut || !x)))
        return sfail(KSC_ERR_ARG, "bad feature arrays");
    for (int i = 0; i < n; ++i) {
        if (nside[i] < 1 || !(fwhm[i] > 0.0) || l_cut[i] < 1 || !(theta_cut[i] > 0.0))
            return sfail(KSC_ERR_ARG, "feature inputs must be positive");
        x[4 * i + 0] = (float)std::log2((double)nside[i]);
        x[4 * i + 1] = (float)std::log(fwhm[i]);
        x[4 * i + 2] = (float)std::log((double)l_cut[i]);
        x[4 * i + 3] = (float)std::log(theta_cut[i]);
    }
    return KSC_OK;
}

int ksc_scan_default_opts(ksc_scan_opts *o) {
    if (!o) return sfail(KSC_ERR_ARG, "null opts");
    o->theta_lo = 30.0 * kArcmin;
    o->theta_hi = 600.0 * kArcmin;
    o->theta_step = 30.0 * kArcmin;
    o->bound = 1e-5;
    o->l_cut_fixed = -1;
    o->linear_steps = 0;
    return KSC_OK;
}

int ksc_scan_split(const double *b_l, int lmax, int nside, const double *cl_in,
                   const ksc_scan_opts *sopts, const ksc_cost_model *cost,
                   const ksc_split_opts *opts, ksc_scan_row *rows, int max_rows, int *n_rows,
                   int *best) {
    if (!b_l || !n_rows || !best) return sfail(KSC_ERR_ARG, "null argument");
    if (lmax < 2 || lmax > 16384) return sfail(KSC_ERR_ARG, "lmax outside 2..16384");
    if (nside < 1 || nside > 8192) return sfail(KSC_ERR_ARG, "nside outside 1..8192");
    ksc_scan_opts so;
    ksc_scan_default_opts(&so);
    if (sopts) so = *sopts;
    if (!(so.theta_step > 0.0) || !(so.theta_lo > 0.0) || so.theta_hi < so.theta_lo ||
        so.theta_hi > kPi || !(so.bound > 0.0) || so.l_cut_fixed >= lmax ||
        so.linear_steps < 0)
        return sfail(KSC_ERR_ARG, "bad scan options");
    ksc_cost_model cm;
    ksc_cost_model_default(&cm);
    if (cost) cm = *cost;
    ksc_split_opts o;
    ksc_default_opts(&o);
    if (opts) o = *opts;
    const int oversample = o.oversample > 0 ? o.oversample : 2;
    const double rcond = o.svd_rcond > 0.0 ? o.svd_rcond : 1e-6;
    const double alpha = o.alpha > 0.0 ? o.alpha : 5.0;
    const int n_con = o.cut_continuity == KSC_CUT_FREE ? 0
                      : (o.cut_continuity == KSC_CUT_C0 ? 1 : 2);
    const int n_theta = (int)std::floor((so.theta_hi - so.theta_lo) / so.theta_step + 1e-9) + 1;
    *n_rows = 0;
    *best = -1;
    std::string msg;
    int rc = KSC_OK;
    // Eq. 6 of the split fitted at (l_cut, theta); < 0 when the fit fails
    auto err = [&](int lc, double th) -> double {
        ksc::FitResult fr;
        const int r = ksc::fit_split_lsq(b_l, lmax, lc, th, cl_in, oversample, rcond, n_con,
                                         &fr, &msg);
        if (r) { rc = r; return -1.0; }
        return ksc::frac_error_eq6(b_l, fr.k_tilde.data(), cl_in, lmax, alpha);
    };
    double best_cost = 0.0;
    try {
        for (int it = 0; it < n_theta; ++it) {
            const double th = so.theta_lo + it * so.theta_step;
            ksc_scan_row row{th, -1, 0.0, 0.0, 0.0};
            if (so.l_cut_fixed >= 0) {
                row.error = err(so.l_cut_fixed, th);
                if (rc) break;
                if (row.error <= so.bound) row.l_cut = so.l_cut_fixed;
            } else {
                int lo = 0, hi = lmax - 1;
                bool found = false;
                if (so.linear_steps > 0) {
                    // ascending pass over evenly spaced l_cut: [lo, hi] becomes the
                    // first step whose upper end meets the bound (lo - 1 failed)
                    const int n = std::min(so.linear_steps, lmax);
                    int prev = -1;
                    for (int i = 1; i <= n && !found; ++i) {
                        const int lc = (int)((long long)(lmax - 1) * i / n);
                        if (lc <= prev) continue;
                        const double e = err(lc, th);
                        if (rc) break;
                        row.error = e;
                        if (e <= so.bound) {
                            lo = prev + 1;
                            hi = lc;
                            found = true;
                        }
                        prev = lc;
                    }
                } else {
                    row.error = err(hi, th);
                    found = row.error <= so.bound;
                }
                if (rc) break;
                if (found) {
                    while (lo < hi) {  // smallest l_cut meeting the bound (bisection)
                        const int mid = (lo + hi) / 2;
                        const double e = err(mid, th);
                        if (rc) break;
                        if (e <= so.bound) hi = mid; else lo = mid + 1;
                    }
                    if (rc) break;
                    row.l_cut = lo;
                    row.error = err(lo, th);
                    if (rc) break;
                }
            }
            const int lc = so.l_cut_fixed >= 0 ? so.l_cut_fixed : row.l_cut;
            ksc_cost_eval(&cm, nside, lc, lmax, th, &row.t_gpu_ms, &row.t_host_ms);
            if (row.l_cut >= 0) {
                const double c = std::max(row.t_gpu_ms, row.t_host_ms);
                if (*best < 0 || c < best_cost) {
                    *best = *n_rows;
                    best_cost = c;
                }
            }
            if (rows && *n_rows < max_rows) rows[*n_rows] = row;
            ++*n_rows;
        }
    } catch (const std::bad_alloc &) {
        return sfail(KSC_ERR_NOMEM, "host allocation in the scan");
    }
    if (rc) return sfail(rc, msg);
    if (*best >= max_rows) *best = -1;  // (the caller's rows array was too short)
    return KSC_OK;
}

} // extern "C"
