// C ABI of libksconv (declared in include/ksconv.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ksc_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(KSC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr double kPi = 3.14159265358979323846;

bool valid_nside(int nside) {
    return nside >= 1 && nside <= 8192 && (nside & (nside - 1)) == 0;
}

template <class T>
cudaError_t dev_upload(T **dst, const T *src, size_t n) {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
    return e;
}

void release(ksc_split *s) {
    if (!s) return;
    cudaFree(s->d_tab);
    cudaFree(s->d_rings);
    cudaFree(s->d_range);
    cudaFree(s->d_items);
    cudaFree(s->d_io);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
}

// Geometry, work list and device table for the real-space part s->c_real.
int finish_split(ksc_split *s, const ksc_split_opts &o) {
    const int nside = s->nside;
    s->chord_cut = 2.0 * std::sin(0.5 * s->theta_cut);
    int n_int = o.n_intervals;
    if (n_int <= 0) {
        double want = 96.0 * s->chord_cut * std::max(s->lmax, 1) / (2.0 * kPi);
        n_int = (int)std::ceil(want);
        n_int = std::max(256, std::min(n_int, ksc::kMaxIntervals));
    }
    if (n_int > ksc::kMaxIntervals) return fail(KSC_ERR_ARG, "n_intervals above 8192");
    s->n_int = n_int;

    ksc::RingGeom g;
    ksc::ring_geometry(nside, &g);
    const int nr = 4 * nside - 1;
    std::vector<ksc::DevRing> rings(nr);
    std::vector<double> th(nr);
    for (int r = 0; r < nr; ++r) {
        rings[r] = {g.z[r], g.s[r], g.len[r], g.start[r], g.phase[r], 0};
        th[r] = std::atan2(g.s[r], g.z[r]);
    }
    // Input-ring range of each output ring: |theta_r - theta_r'| <= theta_cut.
    std::vector<int2> range(nr);
    const double tc = s->theta_cut + 1e-9;
    for (int r = 0; r < nr; ++r) {
        if (s->theta_cut >= kPi) {
            range[r] = make_int2(0, nr - 1);
            continue;
        }
        int lo = (int)(std::lower_bound(th.begin(), th.end(), th[r] - tc) - th.begin());
        int hi = (int)(std::upper_bound(th.begin(), th.end(), th[r] + tc) - th.begin()) - 1;
        range[r] = make_int2(std::max(lo, 0), std::min(hi, nr - 1));
    }
    // Work list: 256-pixel chunks of every ring, ring by ring.
    std::vector<ksc::WorkItem> items;
    s->ring_first_item.assign(nr + 1, 0);
    for (int r = 0; r < nr; ++r) {
        s->ring_first_item[r] = (int)items.size();
        for (int k0 = 0; k0 < g.len[r]; k0 += 256) items.push_back({r, k0});
    }
    s->ring_first_item[nr] = (int)items.size();
    s->n_items = (int)items.size();

    cudaError_t e;
    cudaGetDevice(&s->device);
    if ((e = dev_upload(&s->d_rings, rings.data(), rings.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring table");
    if ((e = dev_upload(&s->d_range, range.data(), range.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring ranges");
    if ((e = dev_upload(&s->d_items, items.data(), items.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");

    // Table build on the GPU: FP64 Legendre recurrence per node (csrc/table.cu).
    double *d_c = nullptr, *d_nodes = nullptr;
    if ((e = dev_upload(&d_c, s->c_real.data(), s->c_real.size())) != cudaSuccess)
        return cuda_fail(e, "upload coefficients");
    if ((e = cudaMalloc(&d_nodes, sizeof(double) * 2 * (n_int + 1))) != cudaSuccess) {
        cudaFree(d_c);
        return cuda_fail(e, "allocate table nodes");
    }
    if ((e = cudaMalloc(&s->d_tab, sizeof(float4) * n_int)) != cudaSuccess) {
        cudaFree(d_c); cudaFree(d_nodes);
        return cuda_fail(e, "allocate table");
    }
    ksc::TableBuild tb{d_c, s->lmax, n_int, s->chord_cut / n_int, s->d_tab, d_nodes};
    e = ksc::launch_table_build(tb, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    cudaFree(d_c);
    cudaFree(d_nodes);
    if (e != cudaSuccess) return cuda_fail(e, "table build");

    ksc::ConvPlan &p = s->plan;
    p.nside = nside;
    p.npix = 12 * nside * nside;
    p.nrings = nr;
    p.d_rings = s->d_rings;
    p.d_range = s->d_range;
    p.d_tab = s->d_tab;
    p.n_int = n_int;
    p.inv_h = (float)(n_int / s->chord_cut);
    p.dc2 = (float)(s->chord_cut * s->chord_cut);
    p.cos_cut = 1.0 - 0.5 * s->chord_cut * s->chord_cut;
    p.domega = (float)(4.0 * kPi / (double)p.npix);
    return KSC_OK;
}

int check_common(int lmax, int nside, double theta_cut) {
    if (lmax < 1 || lmax > 16384) return fail(KSC_ERR_ARG, "lmax outside 1..16384");
    if (!valid_nside(nside)) return fail(KSC_ERR_ARG, "nside must be a power of two in 1..8192");
    if (!(theta_cut > 0.0) || theta_cut > kPi) return fail(KSC_ERR_ARG, "theta_cut outside (0, pi]");
    return KSC_OK;
}

ksc_split_opts resolve_opts(const ksc_split_opts *opts) {
    ksc_split_opts o;
    ksc_default_opts(&o);
    if (opts) {
        o = *opts;
        if (o.oversample <= 0) o.oversample = 2;
        if (!(o.svd_rcond > 0.0)) o.svd_rcond = 1e-6;
        if (!(o.alpha > 0.0)) o.alpha = 5.0;
    }
    return o;
}

int check_maps(const ksc_split *s, const void *a, const void *b) {
    if (!s) return fail(KSC_ERR_ARG, "null split");
    if (!a || !b) return fail(KSC_ERR_ARG, "null map pointer");
    if (a == b) return fail(KSC_ERR_ARG, "in and out must be different buffers");
    return KSC_OK;
}

} // namespace

extern "C" {

int ksc_default_opts(ksc_split_opts *opts) {
    if (!opts) return fail(KSC_ERR_ARG, "null opts");
    opts->mode = KSC_SPLIT_LSQ;
    opts->oversample = 2;
    opts->svd_rcond = 1e-6;
    opts->alpha = 5.0;
    opts->n_intervals = 0;
    return KSC_OK;
}

int ksc_make_split(const double *b_l, int lmax, int nside, int l_cut, double theta_cut,
                   const double *cl_in, const ksc_split_opts *opts, ksc_split **out) {
    if (!out) return fail(KSC_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!b_l) return fail(KSC_ERR_ARG, "null kernel");
    int rc = check_common(lmax, nside, theta_cut);
    if (rc) return rc;
    ksc_split_opts o = resolve_opts(opts);
    if (o.mode != KSC_SPLIT_NONE && (l_cut < 0 || l_cut >= lmax))
        return fail(KSC_ERR_ARG, "l_cut outside 0..lmax-1");
    if (o.mode < KSC_SPLIT_LSQ || o.mode > KSC_SPLIT_NONE) return fail(KSC_ERR_ARG, "bad mode");

    ksc_split *s = new (std::nothrow) ksc_split();
    if (!s) return fail(KSC_ERR_NOMEM, "host allocation");
    s->lmax = lmax; s->nside = nside; s->theta_cut = theta_cut; s->mode = o.mode;
    const int L = lmax + 1;
    try {
        if (o.mode == KSC_SPLIT_LSQ) {
            ksc::FitResult fr;
            std::string msg;
            rc = ksc::fit_split_lsq(b_l, lmax, l_cut, theta_cut, cl_in, o.oversample,
                                    o.svd_rcond, &fr, &msg);
            if (rc) { release(s); return fail(rc, msg); }
            s->l_cut = l_cut;
            s->k_harm = fr.k_harm; s->c_real = fr.c_real; s->k_tilde = fr.k_tilde;
            s->n_unknowns = fr.n_unknowns; s->n_kept = fr.n_kept;
        } else if (o.mode == KSC_SPLIT_SHARP) {
            s->l_cut = l_cut;
            s->k_harm.assign(b_l, b_l + l_cut + 1);
            s->c_real.assign(b_l, b_l + L);
            std::fill(s->c_real.begin(), s->c_real.begin() + l_cut + 1, 0.0);
            s->k_tilde.assign(b_l, b_l + L);  // exact before truncation
        } else {
            s->l_cut = -1;
            s->c_real.assign(b_l, b_l + L);
            s->k_tilde.assign(b_l, b_l + L);
        }
    } catch (const std::bad_alloc &) {
        release(s);
        return fail(KSC_ERR_NOMEM, "host allocation in split fit");
    }
    s->sigma_rms = ksc::sigma_rms_eq2(b_l, s->k_tilde.data(), cl_in, lmax);
    s->frac_error = ksc::frac_error_eq6(b_l, s->k_tilde.data(), cl_in, lmax, o.alpha);
    rc = finish_split(s, o);
    if (rc) { release(s); return rc; }
    *out = s;
    return KSC_OK;
}

int ksc_make_split_real(const double *c_l, int lmax, int nside, double theta_cut,
                        const ksc_split_opts *opts, ksc_split **out) {
    if (!out) return fail(KSC_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!c_l) return fail(KSC_ERR_ARG, "null coefficients");
    int rc = check_common(lmax, nside, theta_cut);
    if (rc) return rc;
    ksc_split_opts o = resolve_opts(opts);
    ksc_split *s = new (std::nothrow) ksc_split();
    if (!s) return fail(KSC_ERR_NOMEM, "host allocation");
    s->lmax = lmax; s->nside = nside; s->theta_cut = theta_cut; s->mode = KSC_SPLIT_NONE;
    s->l_cut = -1;
    s->c_real.assign(c_l, c_l + lmax + 1);
    s->k_tilde = s->c_real;
    rc = finish_split(s, o);
    if (rc) { release(s); return rc; }
    *out = s;
    return KSC_OK;
}

int ksc_split_info(const ksc_split *s, ksc_split_desc *d) {
    if (!s || !d) return fail(KSC_ERR_ARG, "null argument");
    d->lmax = s->lmax; d->l_cut = s->l_cut; d->nside = s->nside; d->mode = s->mode;
    d->n_intervals = s->n_int; d->n_unknowns = s->n_unknowns; d->n_kept = s->n_kept;
    d->theta_cut = s->theta_cut; d->chord_cut = s->chord_cut;
    d->sigma_rms = s->sigma_rms; d->frac_error = s->frac_error; d->n_pairs = s->n_pairs;
    return KSC_OK;
}

int ksc_split_harmonic(const ksc_split *s, double *k) {
    if (!s || !k) return fail(KSC_ERR_ARG, "null argument");
    std::copy(s->k_harm.begin(), s->k_harm.end(), k);
    return KSC_OK;
}

int ksc_split_real_coeffs(const ksc_split *s, double *c) {
    if (!s || !c) return fail(KSC_ERR_ARG, "null argument");
    std::copy(s->c_real.begin(), s->c_real.end(), c);
    return KSC_OK;
}

int ksc_split_model(const ksc_split *s, double *k) {
    if (!s || !k) return fail(KSC_ERR_ARG, "null argument");
    std::copy(s->k_tilde.begin(), s->k_tilde.end(), k);
    return KSC_OK;
}

int ksc_split_table(const ksc_split *s, float *h) {
    if (!s || !h) return fail(KSC_ERR_ARG, "null argument");
    cudaError_t e = cudaMemcpy(h, s->d_tab, sizeof(float4) * s->n_int, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "table download");
    return KSC_OK;
}

int ksc_conv_real(const ksc_split *s, const float *d_in, float *d_out, void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    cudaError_t e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, d_in, d_out, 1,
                                             0, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "conv launch");
    return KSC_OK;
}

int ksc_conv_real_rings(const ksc_split *s, const float *d_in, float *d_out, int ring_lo,
                        int ring_hi, void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    const int nr = 4 * s->nside - 1;
    if (ring_lo < 1 || ring_hi > nr || ring_lo > ring_hi)
        return fail(KSC_ERR_ARG, "ring range outside 1..4 nside - 1");
    const int a = s->ring_first_item[ring_lo - 1], b = s->ring_first_item[ring_hi];
    cudaError_t e = ksc::launch_conv_general(s->plan, s->d_items + a, b - a, d_in, d_out, 1, 0,
                                             nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "conv launch");
    return KSC_OK;
}

int ksc_conv_real_multimap(const ksc_split *s, const float *d_in, float *d_out, int n_maps,
                           void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    if (n_maps < 1 || n_maps > 65535) return fail(KSC_ERR_ARG, "n_maps outside 1..65535");
    cudaError_t e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, d_in, d_out,
                                             n_maps, s->plan.npix, nullptr,
                                             (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "conv launch");
    return KSC_OK;
}

int ksc_conv_real_batch(const ksc_split *const *splits, const float *const *d_in,
                        float *const *d_out, int n, void *stream) {
    if (n < 0 || (n > 0 && (!splits || !d_in || !d_out)))
        return fail(KSC_ERR_ARG, "bad batch arrays");
    for (int i = 0; i < n; ++i) {
        int rc = check_maps(splits[i], d_in[i], d_out[i]);
        if (rc) return rc;
    }
    for (int i = 0; i < n; ++i) {
        int rc = ksc_conv_real(splits[i], d_in[i], d_out[i], stream);
        if (rc) return rc;
    }
    return KSC_OK;
}

int ksc_conv_real_host(const ksc_split *cs, const float *h_in, float *h_out) {
    if (!cs || !h_in || !h_out) return fail(KSC_ERR_ARG, "null argument");
    ksc_split *s = const_cast<ksc_split *>(cs);
    cudaError_t e;
    const size_t bytes = sizeof(float) * (size_t)s->plan.npix;
    if (!s->own_stream) {
        if ((e = cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "stream create");
    }
    if (!s->d_io) {
        if ((e = cudaMalloc(&s->d_io, 2 * bytes)) != cudaSuccess)
            return fail(KSC_ERR_NOMEM, "device buffers for the host path");
    }
    float *din = s->d_io, *dout = s->d_io + s->plan.npix;
    if ((e = cudaMemcpyAsync(din, h_in, bytes, cudaMemcpyHostToDevice, s->own_stream)) != cudaSuccess)
        return cuda_fail(e, "host to device copy");
    e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, din, dout, 1, 0, nullptr,
                                 s->own_stream);
    if (e != cudaSuccess) return cuda_fail(e, "conv launch");
    if ((e = cudaMemcpyAsync(h_out, dout, bytes, cudaMemcpyDeviceToHost, s->own_stream)) != cudaSuccess)
        return cuda_fail(e, "device to host copy");
    if ((e = cudaStreamSynchronize(s->own_stream)) != cudaSuccess)
        return cuda_fail(e, "host path synchronize");
    return KSC_OK;
}

int ksc_count_pairs(ksc_split *s, long long *n_pairs) {
    if (!s || !n_pairs) return fail(KSC_ERR_ARG, "null argument");
    unsigned long long *d_cnt = nullptr;
    cudaError_t e = cudaMalloc(&d_cnt, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "count buffer");
    cudaMemset(d_cnt, 0, sizeof(unsigned long long));
    e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, nullptr, nullptr, 1, 0, d_cnt,
                                 0);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return cuda_fail(e, "pair count");
    s->n_pairs = (long long)h;
    *n_pairs = s->n_pairs;
    return KSC_OK;
}

void ksc_free_split(ksc_split *s) { release(s); }

const char *ksc_status_string(int st) {
    switch (st) {
    case KSC_OK: return "KSC_OK";
    case KSC_ERR_ARG: return "KSC_ERR_ARG";
    case KSC_ERR_NOMEM: return "KSC_ERR_NOMEM";
    case KSC_ERR_CUDA: return "KSC_ERR_CUDA";
    case KSC_ERR_TIMEOUT: return "KSC_ERR_TIMEOUT";
    case KSC_ERR_DEVICE_BOUNDS: return "KSC_ERR_DEVICE_BOUNDS";
    case KSC_ERR_SVD: return "KSC_ERR_SVD";
    case KSC_ERR_UNSUPPORTED: return "KSC_ERR_UNSUPPORTED";
    default: return "KSC_ERR_UNKNOWN";
    }
}

const char *ksc_last_error(void) { return g_last_error.c_str(); }

} // extern "C"
