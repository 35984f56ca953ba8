// Batched persistent launches, CUDA-graph replay and the tile autotuner
// (ksc_batch_* in include/ksconv.h).
//
// A batch is a list of entries, each one map convolved with one split (its own
// nside, beam and theta_cut: a ragged batch).  All entries' work items go into
// one list per (kernel, tile variant) and each list runs as a single persistent
// launch whose CTAs claim items from a device counter.  The list holds the
// entries in decreasing order of total work, each entry's items longest first
// (by the per-ring window cost of its split): the maps in flight stay resident
// in L2 and the launch ends on the smallest items of the smallest entry.  The whole sequence (counter
// reset, belt launches, then gather launches) is captured once as a CUDA graph
// and replayed; the map pointers live in a device entry table that a run
// refreshes only when they change.
//
// The tile variants are the full and half block size of the belt kernel
// (2080 or 1040 outputs per item) and three gather tiles: 256 reflection
// classes per item with 4096-cell weight tables (two CTAs per SM), 128 classes
// with 2048-cell tables (three CTAs per SM; ring pairs needing more cells take
// per-pair weights), and 128 classes with 4096-cell tables (two CTAs per SM).
// Smaller items suit short rings (a 1024-pixel belt ring fills only half of a
// 2080-output item, a ring of 512 pixels has 64 reflection classes).  The autotuner times every
// variant of both kernels on every nside group of the batch, with the caller's
// maps, keeps the fastest of each, and caches the choice per (device, nside,
// l_max, table size, theta_cut) for the rest of the process.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "ksc_internal.h"

namespace {

int bfail(int code, const std::string &msg) {
    ksc::set_last_error(msg);
    return code;
}

int bcuda(cudaError_t e, const char *what) {
    return bfail(KSC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

using TuneKey = std::tuple<int, int, int, int, long long>;  // device, nside, lmax, n_int, theta bits
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;  // -> (belt variant, sym variant)

TuneKey tune_key(const ksc_split *s) {
    long long bits;
    std::memcpy(&bits, &s->theta_cut, sizeof bits);
    return TuneKey(s->device, s->nside, s->lmax, s->n_int, bits);
}

// Untuned default: half blocks only where a belt ring is shorter than a full
// item; the single-map gather tile of that nside.
std::pair<int, int> default_variants(const ksc_split *s) {
    return {4 * s->nside <= ksc::belt_variant_chunk(1) ? 1 : 0,
            ksc::sym_chunk(s->nside) == ksc::sym_variant_chunk(0) ? 0 : 2};
}

struct Launch {
    int kind;     // 0 belt, 1 symmetric gather
    int variant;  // tile variant
    int first, count;  // slice of the item array
    int seg_cap;  // belt only
};

} // namespace

struct ksc_batch {
    int n = 0;
    ksc_batch_opts opts{};
    std::vector<const ksc_split *> splits;   // per entry
    std::vector<const ksc_split *> uniq;     // distinct splits (plan order)
    std::vector<int> plan_of;                // per entry
    std::vector<int> group_of;               // per entry: index into nsides
    std::vector<int> nsides;                 // distinct nside values
    std::vector<std::pair<int, int>> variants;  // per group
    std::vector<int> general;                // entries on the general path (path 1 splits)
    long long n_pairs = 0;                   // in-disc pairs per run, when every split counted them

    ksc::ConvPlan *d_plans = nullptr;
    ksc::BatchEntry *d_entries = nullptr;
    int4 *d_items = nullptr;
    int *d_counters = nullptr;  // one per launch
    int *d_err = nullptr;
    std::vector<Launch> launches;
    int n_items_belt = 0, n_items_sym = 0;

    ksc::BatchEntry *h_entries = nullptr;  // pinned staging of the entry table
    std::vector<ksc::BatchEntry> last;     // entry table now on the device
    cudaEvent_t upload_done = nullptr;
    bool uploaded = false;

    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_stale = true;
};

namespace {

void batch_release_items(ksc_batch *b) {
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    b->d_items = nullptr;
    b->d_counters = nullptr;
    b->launches.clear();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_stale = true;
}

// Reflection classes of northern ring r (0-based; the equator included).
int sym_classes_of(const ksc_split *s, int r) {
    const int L = r < s->nside ? 4 * (r + 1) : 4 * s->nside;  // northern rings and the equator
    const int phase = r < s->nside ? 1 : ((r + 1 - s->nside) % 2 == 0 ? 1 : 0);
    return ksc::sym_classes(L, phase);
}

// Item lists of the entries `sel` under per-group variants; appends launches
// (belt launches first).  Entries on the general path are skipped.
void build_items(const ksc_batch *b, const std::vector<int> &sel,
                 const std::vector<std::pair<int, int>> &vars, std::vector<int4> *items,
                 std::vector<Launch> *launches, int *n_belt, int *n_sym) {
    struct Costed {
        double cost;
        int4 it;
    };
    *n_belt = *n_sym = 0;
    for (int kind = 0; kind < 2; ++kind) {
        for (int v = 0; v < (kind == 0 ? 2 : ksc::sym_variants()); ++v) {
            // per entry: its items, longest first; entries ordered by total cost
            std::vector<std::pair<double, std::vector<Costed>>> per_entry;
            int seg_cap = 0;
            for (int e : sel) {
                const ksc_split *s = b->splits[e];
                if (s->path != 0) continue;
                const std::pair<int, int> var = vars[b->group_of[e]];
                const int nr = s->plan.nrings, eq = (nr - 1) / 2;
                std::vector<Costed> list;
                if (kind == 0) {
                    if (var.first != v || s->n_items_belt == 0) continue;
                    const int chunk = ksc::belt_variant_chunk(v);
                    seg_cap = std::max(seg_cap, ((chunk + s->max_nd + 6 * 13 + 16) + 3) & ~3);
                    for (int r = s->plan.belt_lo; r <= s->plan.belt_hi; ++r) {
                        const int L = 4 * s->nside;
                        for (int k0 = 0; k0 < L; k0 += chunk)
                            list.push_back({std::min(chunk, L - k0) * s->cost_belt[r],
                                            make_int4(e, r, k0, 0)});
                    }
                } else {
                    if (var.second != v) continue;
                    const int chunk = ksc::sym_variant_chunk(v);
                    for (int r = 0; r <= eq; ++r) {
                        if (s->ring_first_sym[r + 1] == s->ring_first_sym[r]) continue;
                        const int n_cls = sym_classes_of(s, r);
                        const double mirror = r == eq ? 1.0 : 2.0;
                        for (int k0 = 0; k0 < n_cls; k0 += chunk)
                            list.push_back({std::min(chunk, n_cls - k0) * s->cost_sym[r] * mirror,
                                            make_int4(e, r, k0, 0)});
                    }
                }
                if (list.empty()) continue;
                std::stable_sort(list.begin(), list.end(),
                                 [](const Costed &x, const Costed &y) { return x.cost > y.cost; });
                double tot = 0.0;
                for (const Costed &c : list) tot += c.cost;
                per_entry.emplace_back(tot, std::move(list));
            }
            if (per_entry.empty()) continue;
            // Entries one after another keep the maps in flight (two or so at a
            // time) resident in L2; interleaving all entries' items strictly
            // longest first would stream every map from HBM for each item.
            std::stable_sort(per_entry.begin(), per_entry.end(),
                             [](const std::pair<double, std::vector<Costed>> &x,
                                const std::pair<double, std::vector<Costed>> &y) {
                                 return x.first > y.first;
                             });
            Launch L;
            L.kind = kind;
            L.variant = v;
            L.first = (int)items->size();
            L.seg_cap = seg_cap;
            for (const auto &pe : per_entry)
                for (const Costed &c : pe.second) items->push_back(c.it);
            L.count = (int)items->size() - L.first;
            launches->push_back(L);
            (kind == 0 ? *n_belt : *n_sym) += L.count;
        }
    }
}

int upload_items(ksc_batch *b, const std::vector<int4> &items, const std::vector<Launch> &launches) {
    batch_release_items(b);
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_items, sizeof(int4) * std::max<size_t>(items.size(), 1))) != cudaSuccess)
        return bfail(KSC_ERR_NOMEM, "batch item list");
    if (!items.empty() &&
        (e = cudaMemcpy(b->d_items, items.data(), sizeof(int4) * items.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return bcuda(e, "batch item upload");
    if ((e = cudaMalloc(&b->d_counters, sizeof(int) * std::max<size_t>(launches.size(), 1))) !=
        cudaSuccess)
        return bfail(KSC_ERR_NOMEM, "batch counters");
    b->launches = launches;
    return KSC_OK;
}

int rebuild(ksc_batch *b) {
    std::vector<int> all(b->n);
    for (int i = 0; i < b->n; ++i) all[i] = i;
    std::vector<int4> items;
    std::vector<Launch> launches;
    build_items(b, all, b->variants, &items, &launches, &b->n_items_belt, &b->n_items_sym);
    return upload_items(b, items, launches);
}

// Enqueue counter reset + launches (+ general-path entries) on st.
int enqueue(ksc_batch *b, const std::vector<Launch> &launches, const int4 *d_items,
            const std::vector<int> *general, cudaStream_t st) {
    cudaError_t e;
    if (!launches.empty() &&
        (e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * launches.size(), st)) != cudaSuccess)
        return bcuda(e, "batch counter reset");
    for (size_t i = 0; i < launches.size(); ++i) {
        const Launch &L = launches[i];
        if (L.kind == 0)
            e = ksc::launch_conv_belt_batch(L.variant, b->d_plans, b->d_entries, d_items + L.first,
                                            L.count, L.seg_cap, b->opts.per_sm_cap, b->d_err,
                                            b->d_counters + i, st);
        else
            e = ksc::launch_conv_sym_batch(L.variant, b->d_plans, b->d_entries, d_items + L.first,
                                           L.count, b->opts.per_sm_cap, b->d_counters + i,
                                           b->d_err, st);
        if (e != cudaSuccess) return bcuda(e, "batch kernel launch");
    }
    if (general) {
        for (int ent : *general) {
            const ksc_split *s = b->splits[ent];
            const ksc::BatchEntry &be = b->last[ent];
            e = ksc::launch_conv_general(s->plan, s->d_items, s->n_items, be.in, be.out, 1, 0, 0,
                                         nullptr, st);
            if (e != cudaSuccess) return bcuda(e, "gather kernel launch");
        }
    }
    return KSC_OK;
}

// Refresh the device entry table when the map pointers changed.
int set_entries(ksc_batch *b, const float *const *d_in, float *const *d_out, cudaStream_t st) {
    std::vector<ksc::BatchEntry> cur(b->n);
    for (int i = 0; i < b->n; ++i) {
        const float *a = d_in[i];
        float *o = d_out[i];
        if (!a || !o) return bfail(KSC_ERR_ARG, "null map pointer");
        if (a == o) return bfail(KSC_ERR_ARG, "in and out must be different buffers");
        if (((uintptr_t)a | (uintptr_t)o) & 15u)
            return bfail(KSC_ERR_ARG, "maps must be 16-byte aligned");
        const ksc_split *s = b->splits[i];
        cur[i] = {a, o, b->plan_of[i], (s->path == 0 && s->n_items_belt > 0) ? 1 : 0};
    }
    bool same = b->uploaded;
    for (int i = 0; same && i < b->n; ++i)
        same = cur[i].in == b->last[i].in && cur[i].out == b->last[i].out;
    if (same) return KSC_OK;
    if (!b->general.empty()) b->graph_stale = true;  // general launches carry the pointers
    cudaError_t e;
    // the staging buffer may still feed the previous upload
    if (b->uploaded && (e = cudaEventSynchronize(b->upload_done)) != cudaSuccess)
        return bcuda(e, "batch entry staging");
    std::memcpy(b->h_entries, cur.data(), sizeof(ksc::BatchEntry) * b->n);
    if ((e = cudaMemcpyAsync(b->d_entries, b->h_entries, sizeof(ksc::BatchEntry) * b->n,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return bcuda(e, "batch entry upload");
    if ((e = cudaEventRecord(b->upload_done, st)) != cudaSuccess)
        return bcuda(e, "batch entry event");
    b->last = cur;
    b->uploaded = true;
    return KSC_OK;
}

int capture(ksc_batch *b) {
    cudaError_t e;
    if (!b->cap_stream &&
        (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bcuda(e, "capture stream");
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bcuda(e, "begin graph capture");
    int rc = enqueue(b, b->launches, b->d_items, &b->general, b->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bcuda(e, "end graph capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(e, "graph instantiate");
    b->graph_stale = false;
    return KSC_OK;
}

void batch_free(ksc_batch *b) {
    if (!b) return;
    batch_release_items(b);
    cudaFree(b->d_plans);
    cudaFree(b->d_entries);
    cudaFree(b->d_err);
    if (b->h_entries) cudaFreeHost(b->h_entries);
    if (b->upload_done) cudaEventDestroy(b->upload_done);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

} // namespace

extern "C" {

int ksc_batch_default_opts(ksc_batch_opts *o) {
    if (!o) return bfail(KSC_ERR_ARG, "null opts");
    o->use_graph = 1;
    o->per_sm_cap = 0;
    return KSC_OK;
}

int ksc_batch_create(const ksc_split *const *splits, int n, const ksc_batch_opts *opts,
                     ksc_batch **out) {
    if (!out) return bfail(KSC_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || !splits) return bfail(KSC_ERR_ARG, "a batch needs n >= 1 splits");
    for (int i = 0; i < n; ++i)
        if (!splits[i]) return bfail(KSC_ERR_ARG, "null split in batch");
    ksc_batch *b = new (std::nothrow) ksc_batch();
    if (!b) return bfail(KSC_ERR_NOMEM, "host allocation");
    ksc_batch_default_opts(&b->opts);
    if (opts) {
        b->opts = *opts;
        if (b->opts.per_sm_cap < 0) b->opts.per_sm_cap = 0;
    }
    b->n = n;
    b->splits.assign(splits, splits + n);
    b->plan_of.resize(n);
    b->group_of.resize(n);
    bool counted = true;
    for (int i = 0; i < n; ++i) {
        const ksc_split *s = splits[i];
        auto it = std::find(b->uniq.begin(), b->uniq.end(), s);
        b->plan_of[i] = (int)(it - b->uniq.begin());
        if (it == b->uniq.end()) b->uniq.push_back(s);
        auto g = std::find(b->nsides.begin(), b->nsides.end(), s->nside);
        b->group_of[i] = (int)(g - b->nsides.begin());
        if (g == b->nsides.end()) {
            b->nsides.push_back(s->nside);
            std::pair<int, int> v = default_variants(s);
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto c = g_tune_cache.find(tune_key(s));
                if (c != g_tune_cache.end()) v = c->second;
            }
            b->variants.push_back(v);
        }
        if (s->path != 0) b->general.push_back(i);
        if (s->n_pairs < 0) counted = false;
        else b->n_pairs += s->n_pairs;
    }
    if (!counted) b->n_pairs = -1;
    std::vector<ksc::ConvPlan> plans;
    for (const ksc_split *s : b->uniq) plans.push_back(s->plan);
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_plans, sizeof(ksc::ConvPlan) * plans.size())) != cudaSuccess ||
        (e = cudaMemcpy(b->d_plans, plans.data(), sizeof(ksc::ConvPlan) * plans.size(),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_entries, sizeof(ksc::BatchEntry) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_err, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(b->d_err, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_entries, sizeof(ksc::BatchEntry) * n)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->upload_done, cudaEventDisableTiming)) != cudaSuccess) {
        batch_free(b);
        return bcuda(e, "batch device state");
    }
    int rc = rebuild(b);
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return KSC_OK;
}

int ksc_batch_run(ksc_batch *b, const float *const *d_in, float *const *d_out, void *stream) {
    ksc::NvtxRange range("ksc_batch_run");
    if (!b || !d_in || !d_out) return bfail(KSC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = set_entries(b, d_in, d_out, st);
    if (rc) return rc;
    if (!b->opts.use_graph) return enqueue(b, b->launches, b->d_items, &b->general, st);
    if (b->graph_stale && (rc = capture(b)) != KSC_OK) return rc;
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return bcuda(e, "graph launch");
    return KSC_OK;
}

int ksc_batch_autotune(ksc_batch *b, const float *const *d_in, float *const *d_out, void *stream,
                       ksc_tune_report *rep) {
    if (!b || !d_in || !d_out) return bfail(KSC_ERR_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = set_entries(b, d_in, d_out, st);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (rep) std::memset(rep, 0, sizeof *rep);
    for (size_t gi = 0; gi < b->nsides.size(); ++gi) {
        std::vector<int> sel;
        for (int i = 0; i < b->n; ++i)
            if (b->group_of[i] == (int)gi && b->splits[i]->path == 0) sel.push_back(i);
        if (sel.empty()) continue;
        const int nv_sym = ksc::sym_variants();
        double ms[2][3] = {{0, 0, 0}, {0, 0, 0}};  // [kind][variant]
        for (int v = 0; v < nv_sym && rc == KSC_OK; ++v) {
            // belt variants 0, 1 and gather variants 0 .. nv_sym - 1 (no belt beyond 1)
            std::vector<std::pair<int, int>> vars(b->nsides.size(), std::make_pair(v, v));
            std::vector<int4> items;
            std::vector<Launch> launches;
            int nb = 0, ns = 0;
            build_items(b, sel, vars, &items, &launches, &nb, &ns);
            // temporary item list and counters, timed per launch (median of 3 after a warm-up)
            int4 *d_items = nullptr;
            int *saved_ctr = b->d_counters;
            int *d_ctr = nullptr;
            cudaError_t e = cudaMalloc(&d_items, sizeof(int4) * std::max<size_t>(items.size(), 1));
            if (e == cudaSuccess)
                e = cudaMalloc(&d_ctr, sizeof(int) * std::max<size_t>(launches.size(), 1));
            if (e == cudaSuccess && !items.empty())
                e = cudaMemcpy(d_items, items.data(), sizeof(int4) * items.size(),
                               cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                rc = bcuda(e, "autotune buffers");
            } else {
                b->d_counters = d_ctr;
                for (size_t li = 0; li < launches.size() && rc == KSC_OK; ++li) {
                    if (launches[li].kind == 0 && v > 1) continue;
                    std::vector<Launch> one(1, launches[li]);
                    std::vector<float> t;
                    for (int rep_i = 0; rep_i < 4 && rc == KSC_OK; ++rep_i) {
                        cudaEventRecord(e0, st);
                        rc = enqueue(b, one, d_items, nullptr, st);
                        cudaEventRecord(e1, st);
                        if (cudaEventSynchronize(e1) != cudaSuccess) rc = bfail(KSC_ERR_CUDA, "autotune sync");
                        float x = 0.0f;
                        cudaEventElapsedTime(&x, e0, e1);
                        if (rep_i > 0) t.push_back(x);
                    }
                    if (!t.empty()) {
                        std::sort(t.begin(), t.end());
                        ms[launches[li].kind][v] += t[t.size() / 2];
                    }
                }
                b->d_counters = saved_ctr;
            }
            cudaFree(d_items);
            cudaFree(d_ctr);
        }
        if (rc) break;
        const bool has_belt = ms[0][0] > 0.0 || ms[0][1] > 0.0;
        int best_sym = 0;
        for (int v = 1; v < nv_sym; ++v)
            if (ms[1][v] < ms[1][best_sym]) best_sym = v;
        std::pair<int, int> best(has_belt && ms[0][1] < ms[0][0] ? 1 : 0, best_sym);
        b->variants[gi] = best;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            for (int i : sel) g_tune_cache[tune_key(b->splits[i])] = best;
        }
        if (rep && gi < 8) {
            rep->n_groups = (int)gi + 1;
            rep->nside[gi] = b->nsides[gi];
            rep->belt_variant[gi] = best.first;
            rep->sym_variant[gi] = best.second;
            for (int v = 0; v < 2; ++v) rep->ms_belt[gi][v] = ms[0][v];
            for (int v = 0; v < 3; ++v) rep->ms_sym[gi][v] = ms[1][v];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    return rebuild(b);
}

int ksc_batch_info(const ksc_batch *b, ksc_batch_desc *d) {
    if (!b || !d) return bfail(KSC_ERR_ARG, "null argument");
    d->n_entries = b->n;
    d->n_splits = (int)b->uniq.size();
    d->n_items_belt = b->n_items_belt;
    d->n_items_sym = b->n_items_sym;
    d->n_launches = (int)b->launches.size() + (int)b->general.size();
    d->use_graph = b->opts.use_graph;
    d->n_pairs = b->n_pairs;
    d->n_groups = (int)b->nsides.size();
    for (int g = 0; g < 8; ++g) {
        d->group_nside[g] = g < d->n_groups ? b->nsides[g] : 0;
        d->group_belt_variant[g] = g < d->n_groups ? b->variants[g].first : 0;
        d->group_sym_variant[g] = g < d->n_groups ? b->variants[g].second : 0;
    }
    return KSC_OK;
}

int ksc_batch_status(ksc_batch *b, void *stream) {
    if (!b) return bfail(KSC_ERR_ARG, "null batch");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(e, "stream synchronize");
    int flag = 0;
    if ((e = cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bcuda(e, "error flag read");
    if (flag) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return bfail(flag, flag == KSC_ERR_TIMEOUT ? "a bounded device wait ran out"
                                                   : "a device-side bounds check fired");
    }
    return KSC_OK;
}

void ksc_batch_free(ksc_batch *b) { batch_free(b); }

} // extern "C"
