// C ABI of libksconv (declared in include/ksconv.h).
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ksc_device.cuh"
#include "ksc_internal.h"
#include "ksc_tc.cuh"

namespace {

// One CTA waits on an mbarrier nothing arrives on (phase 0 never completes); the
// bounded wait runs out and the CTA raises the error flag like a kernel would.
__global__ void wait_probe_kernel(int *err, int max_polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ksc::tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool done = ksc::tc::mbar_wait(&bar, 0u, max_polls);
    if (!done && threadIdx.x == 0) atomicExch(err, KSC_ERR_TIMEOUT);
}

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? KSC_ERR_NOMEM : KSC_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr double kPi = 3.14159265358979323846;

bool valid_nside(int nside) {
    return nside >= 1 && nside <= 8192 && (nside & (nside - 1)) == 0;
}

// Device allocations of one split construction, counted for fault injection.
thread_local int g_alloc_count = 0;

cudaError_t dev_malloc(void **dst, size_t bytes) {
    if (ksc::inject_alloc_fault(++g_alloc_count)) return cudaErrorMemoryAllocation;
    return cudaMalloc(dst, bytes);
}

template <class T>
cudaError_t dev_upload(T **dst, const T *src, size_t n) {
    cudaError_t e = dev_malloc((void **)dst, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
    return e;
}

void release(ksc_split *s) {
    if (!s) return;
    cudaFree(s->d_tab);
    cudaFree(s->d_rings);
    cudaFree(s->d_range);
    cudaFree(s->d_pairs);
    cudaFree(s->d_xinfo);
    cudaFree(s->d_xodd);
    cudaFree(s->d_pair_base);
    cudaFree(s->d_items);
    cudaFree(s->d_items_sym);
    cudaFree(s->d_items_sym_lpt);
    cudaFree(s->d_items_smma);
    cudaFree(s->d_items_smma_lpt);
    cudaFree(s->d_items_mma);
    cudaFree(s->d_ws);
    cudaFree(s->d_items_belt);
    cudaFree(s->d_err);
    cudaFree(s->d_io);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
}

// Geometry, work list and device table for the real-space part s->c_real.
int finish_split(ksc_split *s, const ksc_split_opts &o) {
    const int nside = s->nside;
    g_alloc_count = 0;
    s->chord_cut = 2.0 * std::sin(0.5 * s->theta_cut);
    int n_int = o.n_intervals;
    // ~96 intervals per shortest l_max wavelength; the chord compresses
    // theta by cos(theta/2), so wide cuts need proportionally more
    const double squeeze = std::max(std::cos(0.5 * s->theta_cut), 1e-3);
    const double n_auto = 96.0 * s->chord_cut * std::max(s->lmax, 1) / (2.0 * kPi * squeeze);
    if (n_int <= 0) {
        n_int = (int)std::ceil(n_auto);
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
    // Work lists (ring by ring, with per-ring prefixes for latitude bands):
    //  - all:  256-pixel chunks of every ring (pair counting, fallback);
    //  - belt: belt_chunk()-pixel chunks of belt rings (circulant kernel);
    //  - sym:  first-quarter chunks of northern rings (and the equator) for the
    //          symmetric gather: cap rings, plus belt rings that reach a cap
    //          (every northern ring when the belt kernel is not used).
    const int belt_lo = nside - 1, belt_hi = 3 * nside - 1, eq = 2 * nside - 1;
    std::vector<ksc::WorkItem> items, items_sym;
    std::vector<int2> items_belt;
    s->ring_first_item.assign(nr + 1, 0);
    s->ring_first_sym.assign(nr + 1, 0);
    s->ring_first_belt.assign(nr + 1, 0);
    const int bc = ksc::belt_chunk();
    int max_nd = 0, w_ext = 0;
    for (int r = 0; r < nr; ++r) {
        s->ring_first_item[r] = (int)items.size();
        s->ring_first_sym[r] = (int)items_sym.size();
        s->ring_first_belt[r] = (int)items_belt.size();
        for (int k0 = 0; k0 < g.len[r]; k0 += 256) items.push_back({r, k0});
        const bool belt = r >= belt_lo && r <= belt_hi;
        const bool reaches_cap = range[r].x < belt_lo || range[r].y > belt_hi;
        if (r <= eq && (!belt || reaches_cap || o.path == 1))
            for (int k0 = 0; k0 < ksc::sym_classes(g.len[r], g.phase[r]);
                 k0 += ksc::sym_chunk(nside))
                items_sym.push_back({r, k0});
        if (belt) {
            for (int k0 = 0; k0 < g.len[r]; k0 += bc) items_belt.push_back(make_int2(r, k0));
            // widest circulant window of this ring (same arithmetic as the kernel)
            const int L = g.len[r];
            for (int q = std::max(range[r].x, belt_lo); q <= std::min(range[r].y, belt_hi); ++q) {
                double ss = g.s[r] * g.s[q];
                double cdp = (1.0 - 0.5 * s->chord_cut * s->chord_cut - g.z[r] * g.z[q]) / ss;
                double dphi = cdp <= -1.0 ? 4.0 * kPi : (cdp >= 1.0 ? 0.0 : std::acos(cdp));
                int w = (int)std::ceil(dphi * L / (2.0 * kPi)) + 1;  // same as PairInfo::w
                int n = std::min(2 * w + 1, L);
                max_nd = std::max(max_nd, n);
                w_ext = std::max(w_ext, 2 * w + 1 >= L ? L / 2 : w);
            }
        }
    }
    std::vector<int2> items_mma;
    for (int r = belt_lo; r <= belt_hi; ++r)
        for (int k0 = 0; k0 < g.len[r]; k0 += ksc::belt_mma_block())
            items_mma.push_back(make_int2(r, k0));
    s->n_items_mma = (int)items_mma.size();
    s->w_cap = (max_nd + 2 * 13 + 3) & ~3;
    s->tensor = o.tensor;
    s->mma_ext0 = ((w_ext + 32) + 31) & ~31;
    s->mma_ntiles = (s->mma_ext0 + 4 * nside + (((w_ext + 160) + 31) & ~31)) / 32;
    // the belt tensor kernel needs its weight window in shared memory
    if (s->tensor == 2 && ksc::belt_mma_smem(s->w_cap) > 220u * 1024) s->tensor = 1;
    s->ring_first_item[nr] = (int)items.size();
    s->ring_first_sym[nr] = (int)items_sym.size();
    s->ring_first_belt[nr] = (int)items_belt.size();
    s->n_items = (int)items.size();
    s->n_items_sym = (int)items_sym.size();
    s->n_items_belt = (int)items_belt.size();
    // shared-memory segment: chunk + padded window + alignment, with slack for
    // rounding differences between host and device acos
    const int seg = bc + max_nd + 6 * 13 + 16;
    s->seg_cap = (seg + 3) & ~3;
    s->max_nd = max_nd;
    const bool belt_ok = s->n_items_belt > 0 && 12ull * s->seg_cap <= 200ull * 1024;
    s->path = o.path;
    if (!belt_ok && o.path == 0) {
        // belt windows too wide for shared memory: the general gather does it all
        s->path = 1;
    }
    if (s->path == 1) {
        s->n_items_belt = 0;
        s->seg_cap = 0;
    }

    // Ring-pair geometry (FP64 on the host, once per split).
    std::vector<int> pair_base(nr + 1, 0);
    for (int r = 0; r < nr; ++r) pair_base[r + 1] = pair_base[r] + (range[r].y - range[r].x + 1);
    std::vector<ksc::PairInfo> pairs((size_t)pair_base[nr]);
    std::vector<ksc::XInfo> xinfo((size_t)pair_base[nr]);
    std::vector<ksc::XOdd> xodd((size_t)pair_base[nr]);
    {
        const double dc = s->chord_cut;
        const double cos_cut = 1.0 - 0.5 * dc * dc;
        const double scale2 = ((double)n_int / dc) * ((double)n_int / dc);
        const double dc2 = s->theta_cut >= kPi ? 5.0 : dc * dc;
        // x cells are sized in intervals of the automatic table size, so a coarser
        // user table gets proportionally narrower cells (in its own intervals)
        const double xscale = std::min(1.0, (double)n_int / std::max(n_auto, 1.0));
#pragma omp parallel for schedule(dynamic, 16)
        for (int r = 0; r < nr; ++r) {
            for (int q = range[r].x; q <= range[r].y; ++q) {
                const double dz = g.z[r] - g.z[q];
                const double ds = (g.z[q] - g.z[r]) * (g.z[q] + g.z[r]) / (g.s[r] + g.s[q]);
                const double A = dz * dz + ds * ds;
                const double ss = g.s[r] * g.s[q];
                const int Lq = g.len[q];
                ksc::PairInfo pi;
                const ksc::DF a = ksc::df_from_double(A * scale2);
                const ksc::DF b = ksc::df_from_double(4.0 * ss * scale2);
                const ksc::DF c = ksc::df_from_double(kPi / (2.0 * (double)g.len[r] * (double)Lq));
                pi.Ah = a.h; pi.Al = a.l; pi.Bh = b.h; pi.Bl = b.l; pi.ch = c.h; pi.cl = c.l;
                if (A > dc2 * (1.0 + 1e-6)) {
                    pi.hw = -1.0f;
                    pi.w = -1;
                } else {
                    const double cdp = (cos_cut - g.z[r] * g.z[q]) / ss;
                    const double dphi = cdp <= -1.0 ? 4.0 * kPi : (cdp >= 1.0 ? 0.0 : std::acos(cdp));
                    pi.hw = (float)(dphi * Lq / (2.0 * kPi)) + 1.0f;
                    pi.w = (int)std::ceil(dphi * Lq / (2.0 * kPi)) + 1;
                }
                pairs[(size_t)pair_base[r] + (q - range[r].x)] = pi;
                xinfo[(size_t)pair_base[r] + (q - range[r].x)] =
                    (s->theta_cut >= kPi || o.exact_weights)
                        ? ksc::XInfo{}
                        : ksc::make_xinfo(A * scale2, 4.0 * ss * scale2,
                                          kPi / (2.0 * (double)g.len[r] * (double)Lq),
                                          (double)n_int * (double)n_int, pi.hw, g.len[r], Lq,
                                          xscale);
                xodd[(size_t)pair_base[r] + (q - range[r].x)] =
                    (s->theta_cut >= kPi || o.exact_weights)
                        ? ksc::XOdd{}
                        : ksc::make_xodd(A * scale2, 4.0 * ss * scale2,
                                         kPi / (2.0 * (double)g.len[r] * (double)Lq),
                                         (double)n_int * (double)n_int, pi.hw, g.len[r], Lq,
                                         xscale, ksc::kXCap);
            }
        }
    }

    // Work per output pixel of each ring (window positions over its input
    // rings), for ordering batched work longest first.
    s->cost_belt.assign(nr, 0.0);
    s->cost_sym.assign(nr, 0.0);
    for (int r = 0; r < nr; ++r) {
        const bool belt_r = r >= belt_lo && r <= belt_hi;
        for (int q = range[r].x; q <= range[r].y; ++q) {
            const ksc::PairInfo &pi = pairs[(size_t)pair_base[r] + (q - range[r].x)];
            if (pi.hw < 0.0f) continue;
            const double span = std::min(2.0 * pi.hw + 3.0, (double)g.len[q]);
            const bool belt_q = q >= belt_lo && q <= belt_hi;
            if (s->path == 0 && belt_r && belt_q) s->cost_belt[r] += span;
            else s->cost_sym[r] += span;
        }
    }

    // Share of the symmetric gather's weight evaluations that the dphi tables serve
    // (per northern output ring: reflection classes x window positions per input ring).
    {
        const int eqr = (nr - 1) / 2;
        double all = 0.0, tab = 0.0;
        for (int r = 0; r <= eqr; ++r) {
            const bool belt_r = r >= belt_lo && r <= belt_hi;
            const double cls = (double)ksc::sym_classes(g.len[r], g.phase[r]);
            for (int q = range[r].x; q <= range[r].y; ++q) {
                const size_t ip = (size_t)pair_base[r] + (q - range[r].x);
                if (pairs[ip].hw < 0.0f) continue;
                const bool belt_q = q >= belt_lo && q <= belt_hi;
                if (s->path == 0 && belt_r && belt_q && !items_belt.empty()) continue;
                const double n = cls * std::min(2.0 * pairs[ip].hw + 3.0, (double)g.len[q]);
                all += n;
                if (xodd[ip].nct > 0) tab += n;
            }
        }
        s->frac_tabulated = all > 0.0 ? tab / all : 0.0;
    }

    // The symmetric items longest first, for whole-map launches: CTAs claim items
    // in list order, so the long items start first and the short ones fill the tail.
    // The tensor cap kernel has items of its own size.
    auto lpt = [&](std::vector<ksc::WorkItem> v, int chunk) {
        auto cost = [&](const ksc::WorkItem &w) {
            const int n_cls = ksc::sym_classes(g.len[w.ring], g.phase[w.ring]);
            const int cnt = std::min(chunk, n_cls - w.k0);
            return cnt * s->cost_sym[w.ring] * (w.ring == eq ? 1.0 : 2.0);
        };
        std::stable_sort(v.begin(), v.end(), [&](const ksc::WorkItem &x, const ksc::WorkItem &y) {
            return cost(x) > cost(y);
        });
        return v;
    };
    std::vector<ksc::WorkItem> items_lpt = lpt(items_sym, ksc::sym_chunk(nside));
    // 128-class items of the tensor kernels, ring by ring (with per-ring prefixes
    // for latitude bands) and longest first
    std::vector<ksc::WorkItem> items_smma;
    s->ring_first_smma.assign(nr + 1, 0);
    {
        size_t i = 0;
        for (int r = 0; r < nr; ++r) {
            s->ring_first_smma[r] = (int)items_smma.size();
            if (i < items_sym.size() && items_sym[i].ring == r) {
                const int n_cls = ksc::sym_classes(g.len[r], g.phase[r]);
                for (int k0 = 0; k0 < n_cls; k0 += ksc::sym_mma_chunk())
                    items_smma.push_back({r, k0});
                while (i < items_sym.size() && items_sym[i].ring == r) ++i;
            }
        }
        s->ring_first_smma[nr] = (int)items_smma.size();
    }
    std::vector<ksc::WorkItem> items_smma_lpt = lpt(items_smma, ksc::sym_mma_chunk());
    s->n_items_smma = (int)items_smma.size();
    s->cap_kernel = o.cap_kernel;

    cudaError_t e;
    cudaGetDevice(&s->device);
    if ((e = dev_upload(&s->d_pairs, pairs.data(), pairs.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring-pair table");
    if ((e = dev_upload(&s->d_xinfo, xinfo.data(), xinfo.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring-pair x tables");
    if ((e = dev_upload(&s->d_xodd, xodd.data(), xodd.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring-pair odd-step tables");
    if ((e = dev_upload(&s->d_pair_base, pair_base.data(), pair_base.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring-pair offsets");
    if ((e = dev_upload(&s->d_rings, rings.data(), rings.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring table");
    if ((e = dev_upload(&s->d_range, range.data(), range.size())) != cudaSuccess)
        return cuda_fail(e, "upload ring ranges");
    if ((e = dev_upload(&s->d_items, items.data(), items.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_upload(&s->d_items_sym, items_sym.data(), items_sym.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_upload(&s->d_items_sym_lpt, items_lpt.data(), items_lpt.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_upload(&s->d_items_smma, items_smma.data(), items_smma.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_upload(&s->d_items_smma_lpt, items_smma_lpt.data(), items_smma_lpt.size())) !=
        cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_upload(&s->d_items_belt, items_belt.data(), items_belt.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_upload(&s->d_items_mma, items_mma.data(), items_mma.size())) != cudaSuccess)
        return cuda_fail(e, "upload work list");
    if ((e = dev_malloc((void **)&s->d_err, sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "error flag");
    if ((e = cudaMemset(s->d_err, 0, sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "error flag");

    // Table build on the GPU: FP64 Legendre recurrence per node (csrc/table.cu).
    double *d_c = nullptr, *d_nodes = nullptr;
    if ((e = dev_upload(&d_c, s->c_real.data(), s->c_real.size())) != cudaSuccess)
        return cuda_fail(e, "upload coefficients");
    if ((e = dev_malloc((void **)&d_nodes, sizeof(double) * 2 * (n_int + 1))) != cudaSuccess) {
        cudaFree(d_c);
        return cuda_fail(e, "allocate table nodes");
    }
    if ((e = dev_malloc((void **)&s->d_tab, sizeof(float4) * (n_int + 1))) != cudaSuccess) {
        cudaFree(d_c); cudaFree(d_nodes);
        return cuda_fail(e, "allocate table");
    }
    ksc::TableBuild tb{d_c, s->lmax, n_int, s->chord_cut / n_int, s->d_tab, d_nodes, 1};
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
    p.d_pairs = s->d_pairs;
    p.d_xinfo = s->d_xinfo;
    p.d_xodd = s->d_xodd;
    p.d_pair_base = s->d_pair_base;
    p.d_tab = s->d_tab;
    p.n_int = n_int;
    p.inv_h = (float)(n_int / s->chord_cut);
    p.dc2 = (float)(s->chord_cut * s->chord_cut);
    p.scale2 = ((double)n_int / s->chord_cut) * ((double)n_int / s->chord_cut);
    p.nint2 = (float)((double)n_int * (double)n_int);
    // theta_cut = pi: every pair, whatever the rounding of antipodal chords
    if (s->theta_cut >= kPi) {
        p.dc2 = 5.0f;
        p.nint2 = (float)(1.25 * (double)n_int * (double)n_int);
    }
    p.cos_cut = 1.0 - 0.5 * s->chord_cut * s->chord_cut;
    p.domega = (float)(4.0 * kPi / (double)p.npix);
    p.belt_lo = belt_lo;
    p.belt_hi = belt_hi;
    {
        const ksc::DF c1 = ksc::df_from_double(kPi / (2.0 * 4.0 * nside));
        p.belt_c1h = c1.h;
        p.belt_c1l = c1.l;
    }
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
        if (o.path != 1) o.path = 0;
        if (o.tensor != 1 && o.tensor != 2) o.tensor = 0;
        if (o.cut_continuity < KSC_CUT_C1 || o.cut_continuity > KSC_CUT_FREE)
            o.cut_continuity = KSC_CUT_C1;
        if (o.exact_weights != 1) o.exact_weights = 0;
        if (o.cap_kernel != 1) o.cap_kernel = 0;
    }
    return o;
}

int check_maps(const ksc_split *s, const void *a, const void *b) {
    if (!s) return fail(KSC_ERR_ARG, "null split");
    if (!a || !b) return fail(KSC_ERR_ARG, "null map pointer");
    if (a == b) return fail(KSC_ERR_ARG, "in and out must be different buffers");
    if (((uintptr_t)a | (uintptr_t)b) & 15u)
        return fail(KSC_ERR_ARG, "maps must be 16-byte aligned");
    return KSC_OK;
}

// Tensor-core belt stage for a stack of maps; grows the split's pre-tiled map
// workspace on first use (calls on one split must not overlap on the GPU).
int launch_belt_tensor(const ksc_split *cs, const float *d_in, float *d_out, int n_maps,
                       long long stride, cudaStream_t st) {
    ksc_split *s = const_cast<ksc_split *>(cs);
    const int n_belt = s->plan.belt_hi - s->plan.belt_lo + 1;
    const size_t need = ksc::belt_mma_workspace_floats(n_belt, s->mma_ntiles, n_maps);
    if (s->ws_floats < need) {
        cudaFree(s->d_ws);
        s->d_ws = nullptr;
        s->ws_floats = 0;
        if (cudaMalloc(&s->d_ws, need * sizeof(float)) != cudaSuccess)
            return fail(KSC_ERR_NOMEM, "tensor-path workspace");
        s->ws_floats = need;
    }
    cudaError_t e = ksc::launch_conv_belt_mma(s->plan, s->d_items_mma, s->n_items_mma, s->w_cap,
                                              s->mma_ntiles, s->mma_ext0, s->d_ws, d_in, d_out,
                                              n_maps, stride, s->d_err, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor belt kernel launch");
    return KSC_OK;
}

// The cap stage for the items of northern rings [lo, hi], writing output rings
// [r0, r1]: the map-stack tensor kernel for whole-map stacks, else the FFMA gather
// or the single-map tensor kernel (ksc_split_opts.cap_kernel).  Whole maps take
// the items longest first, bands their rings' items in ring order.
cudaError_t launch_caps(const ksc_split *s, const float *d_in, float *d_out, int n_maps,
                        long long stride, int lo, int hi, int r0, int r1, bool stack,
                        cudaStream_t st) {
    const bool whole = r0 == 0 && r1 == s->plan.nrings - 1;
    const int belt_split = s->n_items_belt > 0 ? 1 : 0;
    if (stack && s->tensor >= 1)
        return ksc::launch_conv_sym_mma(s->plan, s->d_items_smma_lpt, s->n_items_smma, d_in,
                                        d_out, n_maps, stride, belt_split, s->d_err, st);
    if (s->cap_kernel == 1) {
        const int c = s->ring_first_smma[lo], d = s->ring_first_smma[hi + 1];
        const ksc::WorkItem *its = whole ? s->d_items_smma_lpt : s->d_items_smma + c;
        return ksc::launch_conv_sym_tc(s->plan, its, d - c, d_in, d_out, n_maps, stride,
                                       belt_split, r0, r1, s->d_err, st);
    }
    const int c = s->ring_first_sym[lo], d = s->ring_first_sym[hi + 1];
    const ksc::WorkItem *its = whole ? s->d_items_sym_lpt : s->d_items_sym + c;
    return ksc::launch_conv_sym(s->plan, its, d - c, d_in, d_out, n_maps, stride, belt_split,
                                r0, r1, s->d_err, st);
}

// The real-space convolution of output rings [r0, r1] (0-based, inclusive).
// Default path: circulant belt kernel first (writes belt outputs), then the
// symmetric gather (writes cap outputs, adds cap inputs to belt outputs).
// path 1: the general gather alone.
int launch_conv(const ksc_split *s, const float *d_in, float *d_out, int n_maps,
                long long stride, int r0, int r1, cudaStream_t st) {
    ksc::NvtxRange range(n_maps > 1 ? "ksc_conv_real_multimap" : "ksc_conv_real");
    cudaError_t e;
    if (s->path == 1) {
        const int c = s->ring_first_item[r0], d = s->ring_first_item[r1 + 1];
        e = ksc::launch_conv_general(s->plan, s->d_items + c, d - c, d_in, d_out, n_maps,
                                     stride, 0, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "gather kernel launch");
        return KSC_OK;
    }
    const bool whole = r0 == 0 && r1 == s->plan.nrings - 1;
    const bool stack = whole && n_maps >= 16;
    if (stack && s->tensor == 2 && s->n_items_mma > 0) {
        int rc = launch_belt_tensor(s, d_in, d_out, n_maps, stride, st);
        if (rc) return rc;
    } else {
        const int a = s->ring_first_belt[r0], b = s->ring_first_belt[r1 + 1];
        e = ksc::launch_conv_belt(s->plan, s->d_items_belt + a, b - a, s->seg_cap, d_in, d_out,
                                  n_maps, stride, s->d_err, st);
        if (e != cudaSuccess) return cuda_fail(e, "belt kernel launch");
    }
    // northern rings r whose own or mirror ring (nr - 1 - r) lies in the band
    const int nr = s->plan.nrings, eq = (nr - 1) / 2;
    int lo = nr, hi = -1;
    if (r0 <= eq) { lo = r0; hi = std::min(r1, eq); }                // own ring in band
    const int m0 = std::max(0, nr - 1 - r1), m1 = std::min(nr - 1 - r0, eq);
    if (m0 <= m1) { lo = std::min(lo, m0); hi = std::max(hi, m1); }  // mirror in band
    if (lo <= hi) {
        e = launch_caps(s, d_in, d_out, n_maps, stride, lo, hi, r0, r1, stack, st);
        if (e != cudaSuccess) return cuda_fail(e, "symmetric kernel launch");
    }
    return KSC_OK;
}

} // namespace

namespace ksc {
void set_last_error(const std::string &msg) { g_last_error = msg; }

bool inject_alloc_fault(int n) {
    const char *f = std::getenv("KSC_FAULT");
    if (!f || std::strncmp(f, "alloc:", 6) != 0) return false;
    return n == std::atoi(f + 6);
}

XInfo make_xinfo(double A2, double B2, double c, double nint2, float hw, int L, int lq,
                 double scale) {
    XInfo x{};
    // no pair within the cut, or a whole-ring window: no table
    if (hw < 0.0f || 2.0f * hw + 3.0f >= (float)lq || A2 >= nint2 || B2 <= 0.0) return x;
    const double sx2 = (nint2 - A2) / B2;  // sin^2 of x at the cut
    if (sx2 >= 1.0) return x;
    const double xcut = std::asin(std::sqrt(sx2));
    // largest du/dx on [0, xcut]: u^2 = A2 + B2 S, S = sin^2 x, du/dx = B2 sqrt(g(S)) with
    // g = S (1 - S) / (A2 + B2 S), unimodal in S with its peak where B2 S^2 + 2 A2 S = A2
    double dmax;
    if (A2 <= 0.0) {
        dmax = std::sqrt(B2);  // u = sqrt(B2) sin x
    } else {
        double S = (-A2 + std::sqrt(A2 * A2 + A2 * B2)) / B2;
        S = std::min(std::max(S, 0.0), sx2);
        dmax = B2 * std::sqrt(S * (1.0 - S) / (A2 + B2 * S));
    }
    if (!(dmax > 0.0)) return x;
    // the largest |N| within the cut: |N| c <= xcut
    const double nc = std::floor(xcut / c);
    if (nc >= 8388608.0) return x;  // |N| and the quads' reach stay below 2^24
    const int ncut = (int)nc;
    // widest power-of-two cell within kXRho intervals at the steepest point, and no
    // wider than the in-cut range (so that no node lies more than one cell beyond the
    // cut, where the K_r table is extrapolated) ...
    int shift = (int)std::floor(std::log2(scale * kXRho / (dmax * c)));
    shift = std::max(shift, 0);
    while (shift > 0 && std::ldexp(c, shift) * dmax > scale * kXRho) --shift;  // log2 rounding
    while (shift > 0 && (1 << std::min(shift, 30)) > ncut + 1) --shift;
    // ... doubled while the cells (and the reach of an edge quad) would not fit
    auto cells = [&](int sh) { return (ncut >> sh) + 1; };
    while (cells(shift) + kXPad(L, shift) > kXCap && shift < 22) ++shift;
    if (cells(shift) + kXPad(L, shift) > kXCap) return x;
    if (std::ldexp(c, shift) * dmax > scale * kXRhoMax * (1.0 + 1e-12) && shift > 0) return x;
    // integers of in-cut pairs and of positions up to 16 beyond them stay exact in FP32
    if ((double)ncut + 32.0 * (double)L + std::ldexp(1.0, shift) >= 16777216.0) return x;
    x.shift = shift;
    x.ncut = ncut;
    x.ncell = cells(shift);
    return x;
}

XOdd make_xodd(double A2, double B2, double c, double nint2, float hw, int L, int lq,
               double scale, int cap) {
    XOdd x{};
    if (hw < 0.0f || 2.0f * hw + 3.0f >= (float)lq || A2 >= nint2 || B2 <= 0.0) return x;
    const double sx2 = (nint2 - A2) / B2;  // sin^2 of x at the cut
    if (sx2 >= 1.0) return x;
    const double xcut = std::asin(std::sqrt(sx2));
    // largest du/dx on [0, xcut] (as for the power-of-two tables)
    double dmax;
    if (A2 <= 0.0) {
        dmax = std::sqrt(B2);
    } else {
        double S = (-A2 + std::sqrt(A2 * A2 + A2 * B2)) / B2;
        S = std::min(std::max(S, 0.0), sx2);
        dmax = B2 * std::sqrt(S * (1.0 - S) / (A2 + B2 * S));
    }
    if (!(dmax > 0.0)) return x;
    const double nc = std::floor(xcut / c);
    if (nc >= 8388608.0) return x;
    const long long ncut = (long long)nc;
    const long long D = 2LL * lq;
    // widest cell within kXOddRho intervals where the chord changes fastest and no
    // wider than the in-cut range; m the least odd integer giving a cell that narrow
    const double hmax = std::min(scale * kXOddRho / (dmax * c), (double)ncut + 1.0);
    long long m = (long long)std::ceil((double)D / hmax - 1e-9);
    if (m < 1) m = 1;
    if ((m & 1) == 0) ++m;
    auto cells = [&](long long mm) { return (ncut * mm) / D + 1; };  // the zero cell's index
    // wider cells (smaller odd m) while the table and its zero cell would not fit
    while (cells(m) + 1 > cap && m > 1) m -= 2;
    if (cells(m) + 1 > cap) return x;
    const double width = (double)D / (double)m;  // in |N|
    if (width * c * dmax > scale * kXRhoMax * (1.0 + 1e-12)) return x;
    // integers a quarter warp's walk reaches (see XOdd) stay exact
    const double reach = (double)ncut + 48.0 * (double)lq + 40.0 * (double)L;
    if (reach >= 16777216.0 || reach * (double)m + (double)D >= 2147483647.0) return x;
    x.m = (int)m;
    x.nct = (int)cells(m);
    x.off = (int)((long long)x.nct * D - ncut * m - 1);
    x.ncut = (int)ncut;
    const DF cm = df_from_double(c / (double)m);
    x.cmh = cm.h;
    x.cml = cm.l;
    x.hc = (float)(c * width);
    return x;
}
} // namespace ksc

extern "C" {

int ksc_default_opts(ksc_split_opts *opts) {
    if (!opts) return fail(KSC_ERR_ARG, "null opts");
    opts->mode = KSC_SPLIT_LSQ;
    opts->oversample = 2;
    opts->svd_rcond = 1e-6;
    opts->alpha = 5.0;
    opts->n_intervals = 0;
    opts->path = 0;
    opts->tensor = 0;
    opts->cut_continuity = KSC_CUT_C1;
    opts->exact_weights = 0;
    opts->cap_kernel = 0;
    return KSC_OK;
}

int ksc_make_split(const double *b_l, int lmax, int nside, int l_cut, double theta_cut,
                   const double *cl_in, const ksc_split_opts *opts, ksc_split **out) {
    ksc::NvtxRange range("ksc_make_split");
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
            const int n_con = o.cut_continuity == KSC_CUT_FREE ? 0
                              : (o.cut_continuity == KSC_CUT_C0 ? 1 : 2);
            rc = ksc::fit_split_lsq(b_l, lmax, l_cut, theta_cut, cl_in, o.oversample,
                                    o.svd_rcond, n_con, &fr, &msg);
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
    ksc::NvtxRange range("ksc_make_split_real");
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

int ksc_dphi_table_params(double A2, double B2, double c, int n_int, double hw, int lq,
                          double scale, double *out) {
    if (!out || !(c > 0.0) || n_int < 1) return fail(KSC_ERR_ARG, "bad table parameters");
    // the output ring's length from c = pi / (2 L lq)
    const int L = lq > 0 ? (int)std::lround(kPi / (2.0 * c * (double)lq)) : 1;
    const ksc::XInfo x = ksc::make_xinfo(A2, B2, c, (double)n_int * (double)n_int, (float)hw,
                                         std::max(L, 1), lq, scale);
    out[0] = x.ncell > 0 ? std::ldexp(c, x.shift) : 0.0;
    out[1] = (double)x.ncell;
    out[2] = x.ncell > 0 ? (double)x.ncut : 0.0;
    return KSC_OK;
}

int ksc_dphi_odd_params(double A2, double B2, double c, int n_int, double hw, int lq,
                        double scale, int cap, double *out) {
    if (!out || !(c > 0.0) || n_int < 1 || lq < 1 || cap < 2)
        return fail(KSC_ERR_ARG, "bad table parameters");
    const int L = (int)std::lround(kPi / (2.0 * c * (double)lq));
    const ksc::XOdd x = ksc::make_xodd(A2, B2, c, (double)n_int * (double)n_int, (float)hw,
                                       std::max(L, 1), lq, scale, cap);
    out[0] = x.nct > 0 ? c * 2.0 * (double)lq / (double)x.m : 0.0;
    out[1] = (double)x.m;
    out[2] = (double)x.off;
    out[3] = (double)x.nct;
    out[4] = x.nct > 0 ? (double)x.ncut : 0.0;
    return KSC_OK;
}

int ksc_split_info(const ksc_split *s, ksc_split_desc *d) {
    if (!s || !d) return fail(KSC_ERR_ARG, "null argument");
    d->lmax = s->lmax; d->l_cut = s->l_cut; d->nside = s->nside; d->mode = s->mode;
    d->n_intervals = s->n_int; d->n_unknowns = s->n_unknowns; d->n_kept = s->n_kept;
    d->theta_cut = s->theta_cut; d->chord_cut = s->chord_cut;
    d->sigma_rms = s->sigma_rms; d->frac_error = s->frac_error; d->n_pairs = s->n_pairs;
    d->n_pairs_belt = s->n_pairs_belt; d->path = s->path;
    d->frac_tabulated = s->frac_tabulated;
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
    return launch_conv(s, d_in, d_out, 1, 0, 0, s->plan.nrings - 1, (cudaStream_t)stream);
}

int ksc_conv_real_rings(const ksc_split *s, const float *d_in, float *d_out, int ring_lo,
                        int ring_hi, void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    const int nr = 4 * s->nside - 1;
    if (ring_lo < 1 || ring_hi > nr || ring_lo > ring_hi)
        return fail(KSC_ERR_ARG, "ring range outside 1..4 nside - 1");
    return launch_conv(s, d_in, d_out, 1, 0, ring_lo - 1, ring_hi - 1, (cudaStream_t)stream);
}

int ksc_conv_real_multimap(const ksc_split *s, const float *d_in, float *d_out, int n_maps,
                           void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    if (n_maps < 1 || n_maps > 65535) return fail(KSC_ERR_ARG, "n_maps outside 1..65535");
    return launch_conv(s, d_in, d_out, n_maps, s->plan.npix, 0, s->plan.nrings - 1,
                       (cudaStream_t)stream);
}

int ksc_conv_real_batch(const ksc_split *const *splits, const float *const *d_in,
                        float *const *d_out, int n, void *stream) {
    if (n < 0 || (n > 0 && (!splits || !d_in || !d_out)))
        return fail(KSC_ERR_ARG, "bad batch arrays");
    if (n == 0) return KSC_OK;
    for (int i = 0; i < n; ++i) {
        int rc = check_maps(splits[i], d_in[i], d_out[i]);
        if (rc) return rc;
    }
    ksc_batch_opts o;
    ksc_batch_default_opts(&o);
    o.use_graph = 0;
    ksc_batch *b = nullptr;
    int rc = ksc_batch_create(splits, n, &o, &b);
    if (rc) return rc;
    rc = ksc_batch_run(b, d_in, d_out, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    ksc_batch_free(b);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronize");
    return KSC_OK;
}

int ksc_conv_real_host(const ksc_split *cs, const float *h_in, float *h_out) {
    ksc::NvtxRange range("ksc_conv_real_host");
    if (!cs || !h_in || !h_out) return fail(KSC_ERR_ARG, "null argument");
    ksc_split *s = const_cast<ksc_split *>(cs);
    // the split's host-path stream and buffers serve one call at a time
    std::lock_guard<std::mutex> lk(s->host_mu);
    cudaError_t e;
    const size_t bytes = sizeof(float) * (size_t)s->plan.npix;
    if (!s->d_io) {
        g_alloc_count = 0;
        if ((e = dev_malloc((void **)&s->d_io, 2 * bytes)) != cudaSuccess) {
            s->d_io = nullptr;
            return fail(KSC_ERR_NOMEM, "device buffers for the host path");
        }
    }
    if (!s->own_stream) {
        if ((e = cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "stream create");
    }
    float *din = s->d_io, *dout = s->d_io + s->plan.npix;
    if ((e = cudaMemcpyAsync(din, h_in, bytes, cudaMemcpyHostToDevice, s->own_stream)) != cudaSuccess)
        return cuda_fail(e, "host to device copy");
    int rc = launch_conv(s, din, dout, 1, 0, 0, s->plan.nrings - 1, s->own_stream);
    if (rc) return rc;
    if ((e = cudaMemcpyAsync(h_out, dout, bytes, cudaMemcpyDeviceToHost, s->own_stream)) != cudaSuccess)
        return cuda_fail(e, "device to host copy");
    if ((e = cudaStreamSynchronize(s->own_stream)) != cudaSuccess)
        return cuda_fail(e, "host path synchronize");
    return ksc_device_status(s, s->own_stream);
}

int ksc_device_status(const ksc_split *s, void *stream) {
    if (!s) return fail(KSC_ERR_ARG, "null split");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int flag = 0;
    if ((e = cudaMemcpyAsync(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                             (cudaStream_t)stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(e, "error flag read");
    if (flag != 0) {
        // cleared in order on the caller's stream (the flag is shared by every
        // stream that uses the split: clear it where no call on this split runs)
        if ((e = cudaMemsetAsync(s->d_err, 0, sizeof(int), (cudaStream_t)stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize((cudaStream_t)stream)) != cudaSuccess)
            return cuda_fail(e, "error flag clear");
        return fail(flag, "a device-side check fired during an earlier call");
    }
    return KSC_OK;
}

int ksc_probe_wait_timeout(const ksc_split *s, int max_polls, void *stream) {
    if (!s) return fail(KSC_ERR_ARG, "null split");
    if (max_polls <= 0 || max_polls > ksc::tc::kMaxWait) max_polls = ksc::tc::kMaxWait;
    wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(s->d_err, max_polls);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wait probe launch");
    return KSC_OK;
}

int ksc_count_pairs(ksc_split *s, long long *n_pairs) {
    if (!s || !n_pairs) return fail(KSC_ERR_ARG, "null argument");
    unsigned long long *d_cnt = nullptr;
    cudaError_t e = cudaMalloc(&d_cnt, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "count buffer");
    cudaMemset(d_cnt, 0, 2 * sizeof(unsigned long long));
    e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, nullptr, nullptr, 1, 0, 0,
                                 d_cnt, 0);
    if (e == cudaSuccess)
        e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, nullptr, nullptr, 1, 0, 1,
                                     d_cnt + 1, 0);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return cuda_fail(e, "pair count");
    s->n_pairs = (long long)h[0];
    s->n_pairs_belt = (long long)h[1];
    *n_pairs = s->n_pairs;
    return KSC_OK;
}

int ksc_conv_real_multimap_stage(const ksc_split *s, const float *d_in, float *d_out,
                                 int n_maps, int stage, void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    if (n_maps < 1 || n_maps > 65535) return fail(KSC_ERR_ARG, "n_maps outside 1..65535");
    cudaStream_t st = (cudaStream_t)stream;
    const long long stride = s->plan.npix;
    cudaError_t e;
    if (stage == 1) {
        if (s->path == 1) return KSC_OK;
        if (n_maps >= 16 && s->tensor == 2 && s->n_items_mma > 0)
            return launch_belt_tensor(s, d_in, d_out, n_maps, stride, st);
        else
            e = ksc::launch_conv_belt(s->plan, s->d_items_belt, s->n_items_belt, s->seg_cap,
                                      d_in, d_out, n_maps, stride, s->d_err, st);
    } else if (stage == 2) {
        if (s->path == 1)
            e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, d_in, d_out, n_maps,
                                         stride, 0, nullptr, st);
        else
            e = launch_caps(s, d_in, d_out, n_maps, stride, 0, (s->plan.nrings - 1) / 2, 0,
                            s->plan.nrings - 1, n_maps >= 16, st);
    } else {
        return fail(KSC_ERR_ARG, "stage must be 1 or 2");
    }
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    return KSC_OK;
}

int ksc_conv_real_stage(const ksc_split *s, const float *d_in, float *d_out, int stage,
                        void *stream) {
    int rc = check_maps(s, d_in, d_out);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (stage == 1) {
        e = ksc::launch_conv_belt(s->plan, s->d_items_belt, s->n_items_belt, s->seg_cap, d_in,
                                  d_out, 1, 0, s->d_err, st);
    } else if (stage == 2) {
        if (s->path == 1)
            e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, d_in, d_out, 1, 0, 0,
                                         nullptr, st);
        else
            e = launch_caps(s, d_in, d_out, 1, 0, 0, (s->plan.nrings - 1) / 2, 0,
                            s->plan.nrings - 1, false, st);
    } else {
        return fail(KSC_ERR_ARG, "stage must be 1 or 2");
    }
    if (e != cudaSuccess) return cuda_fail(e, "stage launch");
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
    case KSC_ERR_TIMEOUT_UNDRAINED: return "KSC_ERR_TIMEOUT_UNDRAINED";
    default: return "KSC_ERR_UNKNOWN";
    }
}

const char *ksc_last_error(void) { return g_last_error.c_str(); }

} // extern "C"
