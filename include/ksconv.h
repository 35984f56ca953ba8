/*
 * ksconv.h -- C ABI of libksconv, a GB300 (sm_103a) library for the real-space
 * half of the kernel-splitting spherical convolution of Sutter, Wandelt &
 * Elsner, "Using hybrid GPU/CPU kernel splitting to accelerate spherical
 * convolutions" (arXiv:1409.4441).
 *
 * The method (Sec. 2, Fig. 1): a radially symmetric kernel K_l is split into a
 * band-limited harmonic part Khat_l (l <= l_cut), applied by a spherical-
 * harmonic transform, and a compact real-space part Khat_theta (theta <=
 * theta_cut), applied by direct summation on the GPU:
 *
 *     out_i = (4 pi / Npix) * sum_{j : theta_ij <= theta_cut} K_r(theta_ij) m_j
 *
 * over a HEALPix map in RING order.  This library fits the split (Eq. 1-6),
 * tabulates K_r on the GPU and performs that sum.  The harmonic half is the
 * caller's (any SHT library).
 *
 * Conventions
 *   - Angles are radians.  Maps are float32, HEALPix RING order, 12 nside^2
 *     values.  nside is a power of two, 1 <= nside <= 8192.
 *   - Legendre convention: K(z) = sum_l (2l+1)/(4 pi) k_l P_l(z) with
 *     k_l = 2 pi int K(z) P_l(z) dz, so k_0 = 1 is a unit-integral kernel and
 *     convolution multiplies spherical-harmonic coefficients by k_l.
 *   - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()), 16-byte aligned (map data is staged by bulk async copies;
 *     misaligned maps are rejected with KSC_ERR_ARG).  `stream` is a
 *     cudaStream_t passed as void* (NULL = the legacy default stream).  Every ksc_conv_* call is asynchronous on that
 *     stream unless stated otherwise; the caller owns all map buffers and must
 *     keep them alive until the stream has passed the call.
 *   - The library owns a ksc_split and all device memory inside it; release
 *     it with ksc_free_split.  A split may be used from several streams at
 *     once (it is read-only after construction) but must not be freed while
 *     work that uses it is in flight.
 *   - Every entry point returns a status code (0 = success, < 0 = error) and
 *     never throws; ksc_last_error() gives a message for the calling thread.
 */
#ifndef KSCONV_H
#define KSCONV_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define KSC_OK 0
#define KSC_ERR_ARG (-1)           /* invalid argument (sizes, nulls, ranges) */
#define KSC_ERR_NOMEM (-2)         /* host or device allocation failed        */
#define KSC_ERR_CUDA (-3)          /* a CUDA runtime call failed              */
#define KSC_ERR_TIMEOUT (-4)       /* a bounded device wait ran out           */
#define KSC_ERR_DEVICE_BOUNDS (-5) /* a device-side bounds check fired        */
#define KSC_ERR_SVD (-6)           /* the split's SVD did not converge        */
#define KSC_ERR_UNSUPPORTED (-7)   /* valid request this build cannot serve   */
#define KSC_ERR_TIMEOUT_UNDRAINED (-8) /* a bounded wait ran out and copies or
                                      MMAs then in flight did not complete within
                                      the drain's own limit: the kernel's shared
                                      or tensor memory was released (or, for
                                      tensor memory, kept) with them pending   */

/* ---- split construction (Sec. 2, Eq. 1-6) ------------------------------ */
#define KSC_SPLIT_LSQ 0   /* weighted least-squares split, Eq. 3-5 (default) */
#define KSC_SPLIT_SHARP 1 /* Khat_l = K_l (l <= l_cut); real part = the rest */
#define KSC_SPLIT_NONE 2  /* whole kernel in real space, truncated           */

typedef struct ksc_split ksc_split; /* opaque, library-owned */

typedef struct {
    int mode;          /* KSC_SPLIT_*                                          */
    int oversample;    /* real-space unknowns: nodes of an oversample*(lmax+1)
                          point Gauss-Legendre rule inside the cap (z_cut of
                          Eq. 4); default 2                                    */
    double svd_rcond;  /* singular values of the normal matrix A^T W A of
                          Eq. 3 below svd_rcond * max are dropped (those of
                          W^{1/2} A below sqrt(svd_rcond) * max); Sec. 2
                          uses 1e-6; default 1e-6                                */
    double alpha;      /* Eq. 6 numerical-error factor; default 5 (Sec. 3)     */
    int n_intervals;   /* K_r table intervals in the chord d in [0, d_cut];
                          0 = automatic (about 96 per shortest l_max
                          wavelength, at most 8192)                             */
    int path;          /* 0 (default): circulant belt kernel + symmetric gather;
                          1: general ring-pair gather only (reference path)   */
    int tensor;        /* map stacks (ksc_conv_real_multimap, n_maps >= 16):
                          0 (default): FP32 FFMA kernels for every ring pair
                          (per pixel the single-map result, within 1e-6 of
                          the output rms of the FP64 sum);
                          1: the symmetric (cap) ring pairs on the tcgen05
                          tensor cores (TF32 x3, FP32 accumulation of a whole
                          ring pair's window in tensor memory: per pixel
                          within ~3e-5 of the output rms, rms ~2e-6,
                          fractional rms C_l ~1e-6; faster for stacks), the
                          belt ring pairs on the FFMA circulant kernel;
                          2: both kinds of ring pair on the tensor cores
                          (the belt's tensor form is slower than its
                          circulant FFMA form on GB300)                     */
    int cut_continuity; /* LSQ mode: how the fitted real-space kernel meets the
                          cut.  KSC_CUT_FREE is the paper's fit as printed
                          (Sec. 2, Eq. 3-5: K_r truncated at theta_cut, free
                          to jump there; a jump leaves a pixel-sum error on
                          smooth maps of about |K_r(theta_cut)| x boundary
                          pixels).  KSC_CUT_C1 (0, default) and KSC_CUT_C0 are
                          this library's addition to that fit, not part of
                          the paper: the fit also makes K_r vanish at
                          theta_cut, with zero slope (C1) or not (C0), by
                          eliminating the unknowns nearest the cut.  At the
                          nside-2048 5' split (l_cut 1024, 240') the C1 cut
                          gives a fractional rms C_l error of ~5e-6 where the
                          paper's fit gives ~1e-4                           */
    int exact_weights; /* 0 (default): the cap ring pairs' kernel weights come
                          from a per-ring-pair cubic table in dphi / 2 (cells
                          of at most 2-3 intervals of the K_r table, built per
                          work item in shared memory; interpolation error
                          at most 3e-7 of the kernel's peak, rms about 1e-8);
                          1: every weight from the double-float chord and
                          the K_r table                                      */
    int cap_kernel;    /* single maps and stacks of fewer than 16 maps: which
                          kernel sums the cap ring pairs.  0 (default): FP32
                          FFMAs, three reflection classes per thread sharing
                          each staged image value; 1: the tcgen05 tensor
                          cores, each weight and map value split exactly into
                          three BF16 parts and six MMAs per 16 positions
                          (products to FP32 rounding), a fresh accumulator
                          drained every 16 positions into Kahan-folded FP32
                          sums (slower for one map: each weight serves only
                          the 16 symmetry images).  Both use the same
                          weights; their outputs agree to FP32 rounding of
                          the sums                                          */
} ksc_split_opts;

#define KSC_CUT_C1 0
#define KSC_CUT_C0 1
#define KSC_CUT_FREE 2

/* Fill *opts with the defaults listed above. */
int ksc_default_opts(ksc_split_opts *opts);

/*
 * Host-side fault injection (for tests; no GPU fault is made): with the
 * environment variable KSC_FAULT=alloc:N, the N-th device allocation of each
 * split construction (and of the first ksc_conv_real_host call on a split)
 * fails as if the device were out of memory.  The call returns KSC_ERR_NOMEM
 * and releases whatever it had allocated.
 */

/*
 * Fit the split of kernel b_l (l = 0..lmax, host array) for maps of the given
 * nside and build its device table (Sec. 2, Eq. 1-6; Fig. 1 "kernel
 * splitting").  cl_in (host, lmax+1 values, or NULL for a flat spectrum) is
 * the input power spectrum weighting Eq. 2; W = diag((2l+1) C_l^in).
 *   mode LSQ:   minimises Eq. 2 over Khat_l (l <= l_cut) and the z_cut
 *               real-space unknowns; rows l <= l_cut are fitted exactly by
 *               Khat_l and the SVD (with the svd_rcond cut) acts on the
 *               real-space block of rows l > l_cut.
 *   mode SHARP: Khat_l = b_l for l <= l_cut; real part = sum over l > l_cut.
 *   mode NONE:  l_cut is ignored (no harmonic part); real part = b_l.
 * Requires 1 <= lmax <= 16384, 0 <= l_cut < lmax (LSQ/SHARP),
 * 0 < theta_cut <= pi.  Runs host FP64 code (OpenMP) and one table-building
 * kernel on the current device; synchronous.  On success *out owns a new split.
 * Errors: KSC_ERR_ARG, KSC_ERR_NOMEM, KSC_ERR_SVD, KSC_ERR_CUDA.
 */
int ksc_make_split(const double *b_l, int lmax, int nside, int l_cut,
                   double theta_cut, const double *cl_in,
                   const ksc_split_opts *opts, ksc_split **out);

/*
 * Build a split whose real-space part is given directly by its Legendre
 * coefficients c_l (l = 0..lmax, host): K_r(theta) = sum_l (2l+1)/(4 pi) c_l
 * P_l(cos theta) for theta <= theta_cut, 0 beyond (the table of Sec. 3,
 * Fig. 4).  No harmonic part.  Same requirements and errors as above.
 */
int ksc_make_split_real(const double *c_l, int lmax, int nside,
                        double theta_cut, const ksc_split_opts *opts,
                        ksc_split **out);

typedef struct {
    int lmax, l_cut, nside, mode, n_intervals, n_unknowns, n_kept;
    double theta_cut;     /* radians                                          */
    double chord_cut;     /* 2 sin(theta_cut / 2)                             */
    double sigma_rms;     /* Eq. 2 of the fitted split                        */
    double frac_error;    /* Eq. 6 estimate with opts.alpha                   */
    long long n_pairs;    /* ordered in-disc pixel pairs (one map), or -1     */
    long long n_pairs_belt; /* of which both pixels lie in the belt, or -1    */
    int path;             /* kernel path in use (see ksc_split_opts.path)     */
    double frac_tabulated; /* share of the symmetric gather's weight
                              evaluations (window positions x reflection
                              classes) served by dphi tables (0 with
                              exact_weights = 1)                              */
} ksc_split_desc;

/* Describe a split (host struct, filled synchronously). */
int ksc_split_info(const ksc_split *s, ksc_split_desc *out);
/* Copy out the harmonic part Khat_l, l = 0..l_cut (host array). */
int ksc_split_harmonic(const ksc_split *s, double *k_harm);
/* Copy out the real-space Legendre coefficients c_l, l = 0..lmax (host). */
int ksc_split_real_coeffs(const ksc_split *s, double *c_l);
/* Copy out the fitted kernel K~_l = Khat_l + P Khat_theta (Eq. 1), l = 0..lmax. */
int ksc_split_model(const ksc_split *s, double *k_tilde);
/* Copy the device table to host: 4 floats (a0..a3) per interval; on interval
 * k, K(d) = a0 + t(a1 + t(a2 + t a3)), t = d/h - k, h = chord_cut/n_intervals. */
int ksc_split_table(const ksc_split *s, float *host_coeffs);

/* ---- the real-space convolution (the hot path) ------------------------- */
/*
 * out = real-space convolution of `in` with the split's K_r (both device
 * arrays of 12 nside^2 floats, nside as given to the split; in != out).
 * Asynchronous on `stream`.  Each call takes a few bytes of work-claim
 * counters from the device's default stream-ordered memory pool
 * (cudaMallocAsync / cudaFreeAsync on `stream`), so calls on several streams
 * may overlap and a call captured into a CUDA graph holds its own counters.
 * Errors: KSC_ERR_ARG, KSC_ERR_CUDA.
 */
int ksc_conv_real(const ksc_split *s, const float *d_in, float *d_out,
                  void *stream);

/*
 * Latitude band: write only output rings ring_lo..ring_hi (1-based HEALPix
 * ring numbers, 1 <= ring_lo <= ring_hi <= 4 nside - 1); other outputs are
 * untouched.  Reads whatever input rings the band needs (Sec. 4 latitude
 * bands with theta_cut overlap).  Results are bit-identical to the same rings
 * of ksc_conv_real.
 */
int ksc_conv_real_rings(const ksc_split *s, const float *d_in, float *d_out,
                        int ring_lo, int ring_hi, void *stream);

/*
 * n_maps maps sharing one split: d_in and d_out are [n_maps][12 nside^2]
 * device arrays (map-major).  Asynchronous.  By default every map runs the
 * single-map kernels (same results, one launch per stage for the stack).
 * With opts.tensor = 1 and n_maps >= 16 the cap ring pairs run on the tensor
 * cores (each kernel weight evaluated once for a group of 8 maps and their 16
 * symmetry images; per pixel within ~3e-5 of the output rms of the FFMA
 * result, see ksc_split_opts.tensor).  With opts.tensor = 2 the belt ring pairs
 * also run on the tensor cores, through a per-split workspace (the map stack
 * pre-split into TF32 tiles, about 2.6x the input size) allocated on the
 * first such call and reused; multi-map calls on such a split must not
 * overlap on the GPU.
 */
int ksc_conv_real_multimap(const ksc_split *s, const float *d_in,
                           float *d_out, int n_maps, void *stream);

/*
 * A ragged batch: n independent convolutions (each its own split, hence its
 * own nside, beam and theta_cut) in one call; splits, d_in and d_out are
 * host arrays of n entries.  Runs a transient ksc_batch (below, without graph
 * capture) and releases it before returning: synchronous on `stream`.  For
 * repeated batches create a ksc_batch once and call ksc_batch_run.
 */
int ksc_conv_real_batch(const ksc_split *const *splits,
                        const float *const *d_in, float *const *d_out, int n,
                        void *stream);

/* ---- batched persistent launches, CUDA graphs, autotuned tiles --------- */
/*
 * A ksc_batch holds n entries, entry i = one map convolved with splits[i]
 * (entries may repeat a split: a stack of maps under one kernel; or mix
 * nside, beam and theta_cut: a ragged batch).  The work items of all entries
 * are merged into one list per kernel and tile variant (entries in decreasing
 * order of work, each entry's items longest first) and each list runs as ONE
 * persistent launch whose CTAs claim items from a device counter (so short
 * maps fill the tail of long ones).  With use_graph the launch sequence is
 * captured once as a CUDA graph and replayed.  Results equal those of
 * ksc_conv_real on each entry to FP32 rounding (the batch kernels are separate
 * instantiations, free to contract multiply-adds differently, and the
 * half-size gather tile regroups the FP32 partial sums); repeated runs of a
 * batch are bitwise reproducible.
 * The splits must outlive the batch.  Batches are not thread-safe: one run at
 * a time per batch (runs of one batch on one stream are ordered).
 */
typedef struct ksc_batch ksc_batch; /* opaque, library-owned */

typedef struct {
    int use_graph;   /* 1 (default): capture the launches once as a CUDA graph
                        and replay it; 0: enqueue the launches on each run   */
    int per_sm_cap;  /* resident CTAs per SM; 0 (default) = occupancy limit  */
} ksc_batch_opts;

int ksc_batch_default_opts(ksc_batch_opts *opts);

/* Build a batch (host work lists, device tables; synchronous).  Tile variants
 * come from earlier ksc_batch_autotune results of this process for the same
 * device, nside, lmax, table size and theta_cut, else a default (half-size
 * belt items where a belt ring has at most 1040 pixels).
 * Errors: KSC_ERR_ARG, KSC_ERR_NOMEM, KSC_ERR_CUDA. */
int ksc_batch_create(const ksc_split *const *splits, int n,
                     const ksc_batch_opts *opts, ksc_batch **out);

/* Convolve every entry: d_in[i], d_out[i] are device maps of entry i (host
 * arrays of n pointers, same rules as ksc_conv_real).  Asynchronous on
 * `stream`; the pointer table is re-uploaded only when it changed since the
 * previous run.  Errors: KSC_ERR_ARG, KSC_ERR_CUDA. */
int ksc_batch_run(ksc_batch *b, const float *const *d_in, float *const *d_out,
                  void *stream);

typedef struct {
    int n_groups;              /* nside groups tuned (at most 8 reported)    */
    int nside[8];
    int belt_variant[8];       /* 0: 2080-output belt items, 1: 1040         */
    int sym_variant[8];        /* gather items: 0: 256 classes (4096-cell
                                  weight tables, 2 CTAs per SM), 1: 128
                                  classes (2048 cells, 3 CTAs per SM), 2: 128
                                  classes (4096 cells, 2 CTAs per SM)        */
    double ms_belt[8][2];      /* median launch time of each belt variant    */
    double ms_sym[8][3];       /* median launch time of each gather variant  */
} ksc_tune_report;

/* The autotuner: for every nside group of the batch, time each tile variant
 * of the belt kernel and of the symmetric gather on the given maps (a warm-up
 * and three timed launches each, CUDA events on `stream`), keep the faster of
 * each, rebuild the work lists, and remember the choice for later batches in
 * this process.  Synchronous.  d_out holds no defined result afterwards (the
 * gather adds into it repeatedly): run the batch again.  rep may be NULL. */
int ksc_batch_autotune(ksc_batch *b, const float *const *d_in,
                       float *const *d_out, void *stream, ksc_tune_report *rep);

typedef struct {
    int n_entries, n_splits, n_groups;
    int n_items_belt, n_items_sym;  /* items over all persistent launches   */
    int n_launches;                 /* kernel launches per run              */
    int use_graph;
    long long n_pairs;              /* in-disc pairs per run, or -1 when a
                                       split has not counted its pairs      */
    int group_nside[8], group_belt_variant[8], group_sym_variant[8];
} ksc_batch_desc;

int ksc_batch_info(const ksc_batch *b, ksc_batch_desc *out);

/* Synchronize `stream` and report device-side errors raised by runs of this
 * batch (as ksc_device_status does for a split); clears the flag. */
int ksc_batch_status(ksc_batch *b, void *stream);

/* Release a batch (NULL is a no-op); its runs must have completed. */
void ksc_batch_free(ksc_batch *b);

/*
 * End-to-end convenience: host map in, host map out (12 nside^2 floats each),
 * through library-owned device buffers and the split's own stream (both
 * created by the first call).  Synchronous.  Calls on one split from several
 * host threads take turns (the buffers are the split's); calls on different
 * splits run concurrently.  Errors: KSC_ERR_ARG, KSC_ERR_NOMEM, KSC_ERR_CUDA.
 */
int ksc_conv_real_host(const ksc_split *s, const float *h_in, float *h_out);

/*
 * One stage of ksc_conv_real, for profiling and custom scheduling: stage 1 =
 * the circulant kernel for belt-belt ring pairs (writes the belt outputs; a
 * no-op on path 1), stage 2 = the gather for every other pair (writes cap
 * outputs and, after stage 1, adds the cap inputs of belt outputs).  Stage 1
 * then stage 2 on one stream equals ksc_conv_real bit for bit.
 */
int ksc_conv_real_stage(const ksc_split *s, const float *d_in, float *d_out,
                        int stage, void *stream);

/* The same two stages for a stack of n_maps maps ([n_maps][Npix] device
 * arrays); each stage uses the tensor kernel under the same rule as
 * ksc_conv_real_multimap.  Stage 1 then stage 2 equals that call bit for bit. */
int ksc_conv_real_multimap_stage(const ksc_split *s, const float *d_in,
                                 float *d_out, int n_maps, int stage,
                                 void *stream);

/* Count ordered in-disc pixel pairs on the device (synchronous); also stored
 * in the split (with the belt-belt subset) and reported by ksc_split_info. */
int ksc_count_pairs(ksc_split *s, long long *n_pairs);

/*
 * The dphi weight table the symmetric gather builds for one ring pair, as the
 * library sizes it (host arithmetic only, no device work; for inspection).
 * For output ring r (L pixels) and input ring q (lq pixels) the squared chord in
 * K_r-table units is A2 + B2 sin^2 x, x = dphi / 2 = |N| c, c = pi / (2 L lq),
 * n_int the table's intervals (the cut is A2 + B2 sin^2 x <= n_int^2); hw is
 * the gather's window half-width in input pixels (< 0: no pair within the cut;
 * 2 hw + 3 >= lq: the window is the whole ring, which gets no table), scale
 * = min(1, n_int / automatic n_int).  out[0] = cell width in x (radians),
 * out[1] = number of cells (0: per-pair chord weights), out[2] = the largest
 * |N| within the cut.  KSC_ERR_ARG for a null out, c <= 0 or n_int < 1.
 */
int ksc_dphi_table_params(double A2, double B2, double c, int n_int, double hw,
                          int lq, double scale, double *out);

/*
 * Host-only view (no device work) of the odd-step weight table the lockstep
 * symmetric gather builds for one ring pair, from the same inputs as
 * ksc_dphi_table_params plus the cells a CTA holds (cap, zero cell included).
 * The table tabulates the ring pair's weight in the exact pixel-pair integer
 * |N| in cubic cells of 2 lq / m integers, m odd, at the rational position
 * P = (|N| m + off) / (2 lq): cells 0 .. nct-1 cover |N| <= ncut (the cut),
 * cell nct is zero.  out[0] = cell width in x = dphi / 2 (radians), out[1] = m,
 * out[2] = off, out[3] = nct (0: no table), out[4] = ncut.  Errors: KSC_ERR_ARG.
 */
int ksc_dphi_odd_params(double A2, double B2, double c, int n_int, double hw, int lq,
                        double scale, int cap, double *out);

/*
 * Synchronize `stream` and report device-side errors raised by earlier calls
 * on this split: KSC_ERR_TIMEOUT when a bounded wait inside a kernel ran out
 * (the kernel stopped early and its output is incomplete),
 * KSC_ERR_TIMEOUT_UNDRAINED when, in addition, copies or MMAs then in flight
 * outlived the kernel's bounded drain, KSC_ERR_DEVICE_BOUNDS when a device-side
 * check of the kernels' index invariants fired.  The flag is shared by every
 * stream that uses the split; it is read and cleared in order on `stream`, so
 * call this where no other work on the split is in flight.  KSC_OK otherwise.
 */
int ksc_device_status(const ksc_split *s, void *stream);

/*
 * Exercise the bounded-wait failure path on `stream`: one CTA waits on a
 * shared-memory mbarrier that no thread ever arrives on, with the same bounded
 * poll loop as the kernels; when max_polls tries have run out (max_polls <= 0:
 * the kernels' own limit, 2^22 tries, about 16 s on a GB300) it raises this
 * split's device error flag as a kernel would, and returns.  Nothing hangs or
 * faults: the next ksc_device_status reports KSC_ERR_TIMEOUT and clears the
 * flag, and the context stays usable.  Asynchronous; errors: KSC_ERR_ARG,
 * KSC_ERR_CUDA.
 */
int ksc_probe_wait_timeout(const ksc_split *s, int max_polls, void *stream);

/*
 * Allocation-free table build (the paper has no counterpart: this serves
 * callers that cannot allocate device memory where they need a table, such as
 * code under a caching allocator or a fixed memory budget that owns all
 * device memory, real-time loops that cannot afford cudaMalloc's implicit
 * synchronisation, or work issued during CUDA stream capture).
 * Builds the same K_r table as ksc_make_split_real (see ksc_split_table for
 * the layout): d_c = lmax+1 real-space Legendre coefficients (device, FP64),
 * d_table = n_intervals * 4 floats (device, 16-byte aligned), both owned by
 * the caller.  Asynchronous on `stream`; calls no allocator.  Its node scratch
 * is a built-in device array sized for n_intervals <= 8192 (131 kB held on
 * every device that loads the library until exit); larger n_intervals is
 * rejected with KSC_ERR_ARG.  Calls share that array: calls that overlap on
 * the GPU race.  A call made outside stream capture looks up the array's
 * address (which follows a reset of the device's context); a call made during
 * capture uses the address of the last call outside capture on that device, so
 * make one call before any capture (KSC_ERR_ARG otherwise).
 * Errors: KSC_ERR_ARG, KSC_ERR_CUDA, KSC_ERR_UNSUPPORTED (device index > 63).
 */
int ksc_build_table_noalloc(const double *d_c, int lmax, double theta_cut,
                            int n_intervals, float *d_table, void *stream);

/* ---- the harmonic half on the GPU (optional; Fig. 1's CPU half) ------- */
/*
 * Spherical-harmonic transforms of HEALPix RING maps up to l_max = lmax (the
 * split's l_cut for the harmonic half), m <= lmax, real fields:
 *   synthesis  m_p = sum_l [a_l0 Y_l0(p) + 2 Re sum_{m>0} a_lm Y_lm(p)],
 *   analysis   a_lm = (4 pi / Npix) sum_p m_p conj(Y_lm(p))  (equal-weight
 *              quadrature, the paper's pixel-sum convention),
 * with Y_lm = lambda_lm(cos theta) e^{i m phi}, lambda_lm normalised associated
 * Legendre functions without the Condon-Shortley phase.  a_lm are complex
 * doubles (re, im interleaved) in m-major order: index(l, m) = m (2 lmax + 1 - m)
 * / 2 + l, m = 0..lmax, l = m..lmax; (lmax + 1)(lmax + 2) / 2 entries.
 * Legendre recurrences in FP64 (scaled against underflow near the poles), ring
 * sums in FP32.  Device pointers; asynchronous on `stream`; scratch from the
 * stream-ordered allocator.  nside a power of two <= 8192, 0 <= lmax <= 4 nside.
 * Errors: KSC_ERR_ARG, KSC_ERR_NOMEM, KSC_ERR_CUDA.
 */
int ksc_sht_alm2map(int nside, int lmax, const double *d_alm, float *d_map,
                    void *stream);
int ksc_sht_map2alm(int nside, int lmax, const float *d_map, double *d_alm,
                    void *stream);
/*
 * The harmonic half of the split: d_out = synthesis(Khat_l a_lm) with a_lm the
 * analysis of d_in to l_cut (Fig. 1's CPU half, here on the GPU); add != 0
 * adds it to d_out instead (e.g. onto ksc_conv_real's result: the whole split
 * convolution).  KSC_ERR_ARG for a split without a harmonic part.
 */
int ksc_conv_harmonic(const ksc_split *s, const float *d_in, float *d_out, int add,
                      void *stream);

/* ---- split planning: cost models and the scan of Sec. 2 ---------------- */
/*
 * Cost of the two halves of a split convolution (Sec. 2, Eq. 7-8, refitted for
 * this library; host arithmetic only):
 *   t_gpu  = gpu_ms0 + (gpu_ms_per_tpair + gpu_ms_per_tpair_ring * 1000 / nside)
 *            * P * 1e-12,  P = ksc_cost_pairs(nside, theta_cut)
 *            (the real-space half costs a fixed amount per in-disc pixel pair, plus
 *            a per-ring-pair overhead -- table build, staging -- which at a given
 *            pair count grows as rings shorten, ~1/nside; the paper's Eq. 7 is
 *            linear in theta_cut for its GTX 480 code);
 *   t_host = host_ms0 + host_ms_eq8 * l_cut^2 l_max / 4096^3
 *            (Eq. 8's form for the harmonic half; the paper's host_ms_eq8 = 160e3
 *            on one 2.8 GHz core).
 */
typedef struct {
    double gpu_ms0, gpu_ms_per_tpair;
    double host_ms0, host_ms_eq8;
    double gpu_ms_per_tpair_ring; /* default 0 (the nside-2048 benchmark's model) */
} ksc_cost_model;

/* In-disc pixel pairs of a map, Npix^2 (1 - cos theta_cut) / 2, Npix = 12 nside^2. */
double ksc_cost_pairs(int nside, double theta_cut);
/* GPU: this library on one GB300 (the nside-2048 benchmark: 259 ms for
 * 3.09e12 pairs); host: Eq. 8 as printed.  Refit both for the machine at hand. */
int ksc_cost_model_default(ksc_cost_model *m);
/* t_gpu and t_host (ms) of one split (l_cut < 0: no harmonic half, t_host = 0);
 * either output may be NULL. */
int ksc_cost_eval(const ksc_cost_model *m, int nside, int l_cut, int lmax,
                  double theta_cut, double *t_gpu_ms, double *t_host_ms);
/* Least-squares fits (in relative error, every coefficient >= 0) of the three GPU
 * terms to n >= 3 measured real-space convolution times (with a single nside the
 * two pair terms cannot be told apart: the ring term is then 0), and of the two
 * host terms to n >= 2 measured harmonic-half times; each updates only its own
 * half of *m.  KSC_ERR_ARG for non-positive times or degenerate data. */
int ksc_cost_fit_gpu(const int *nside, const double *theta_cut, const double *t_ms,
                     int n, ksc_cost_model *m);
int ksc_cost_fit_host(const int *l_cut, const int *lmax, const double *t_ms, int n,
                      ksc_cost_model *m);

/* The surrogate's inputs for n splits: x[i] = (log2 nside, ln FWHM[rad],
 * ln l_cut, ln theta_cut[rad]) as floats (x: n x 4, host).  KSC_ERR_ARG for
 * non-positive inputs. */
int ksc_split_features(int n, const int *nside, const double *fwhm,
                       const int *l_cut, const double *theta_cut, float *x);

typedef struct {
    double theta_lo, theta_hi, theta_step; /* radians; default 30' .. 600' in 30'
                                              steps (Table 1's cuts are multiples
                                              of 30')                          */
    double bound;      /* Eq. 6 bound on the fractional error; default 1e-5      */
    int l_cut_fixed;   /* -1 (default): search l_cut per theta_cut;
                          >= 0: only theta_cut is scanned, at this l_cut        */
    int linear_steps;  /* 0 (default): the l_cut search is Sec. 2's binary search
                          over 0..l_max-1 (it takes the error as falling with
                          l_cut); n > 0: first an ascending pass over n evenly
                          spaced l_cut values, then bisection inside the first
                          step that meets the bound -- for errors that are not
                          monotone in l_cut (with the SVD cut active they are
                          not, beyond about l_max / 2).  Costs up to n + log2
                          (l_max / n) split fits per theta_cut.               */
} ksc_scan_opts;

typedef struct {
    double theta_cut;  /* radians                                               */
    int l_cut;         /* smallest l_cut meeting the bound, or -1 if none       */
    double error;      /* Eq. 6 at (l_cut, theta_cut); with no l_cut meeting the
                          bound: at l_max - 1 (or at l_cut_fixed)              */
    double t_gpu_ms, t_host_ms; /* the cost model at that split                 */
} ksc_scan_row;

int ksc_scan_default_opts(ksc_scan_opts *o);
/*
 * Sec. 2's scanning strategy for kernel b_l (l = 0..lmax) on maps of nside: for
 * each theta_cut of the grid, a search for the smallest l_cut whose least-
 * squares split (fitted as ksc_make_split does, with split_opts; NULL =
 * defaults) meets bound in Eq. 6 (with split_opts->alpha; a binary search as in
 * Sec. 2, or the linear pass of scan->linear_steps); then the candidate of least
 * max(t_gpu, t_host) under `cost` (NULL = ksc_cost_model_default), the two halves
 * running concurrently (Fig. 1).  rows (max_rows entries, may be NULL) receives
 * one row per theta_cut, *n_rows their number, *best the index of the chosen row
 * (-1: no split meets the bound, or it did not fit in rows).  Host FP64 only
 * (no GPU); synchronous; about one split fit per binary-search step.
 * Errors: KSC_ERR_ARG, KSC_ERR_NOMEM, KSC_ERR_SVD.
 */
int ksc_scan_split(const double *b_l, int lmax, int nside, const double *cl_in,
                   const ksc_scan_opts *scan, const ksc_cost_model *cost,
                   const ksc_split_opts *split_opts, ksc_scan_row *rows,
                   int max_rows, int *n_rows, int *best);

/* ---- surrogate split selector (learned error / cost model) ------------ */
/*
 * A 4-64-64-2 multilayer perceptron (tanh hidden layers, FP32) that predicts,
 * for a split described by x = (log2 nside, ln FWHM[rad], ln l_cut,
 * ln theta_cut[rad]), y = (log10 eps_C, log10 t_conv[ms]): the measured
 * fractional-rms C_l error of the split convolution and the GPU time of its
 * real-space part.  It stands beside the paper's Eq. 6 error estimate and
 * Eq. 7-8 cost models (Sec. 2 scan) so a split meeting an error bound can be
 * chosen without trial runs; a measured run remains the final check.  It is trained
 * on the GPU by the library's own forward / backward / Adam kernels (the paper
 * has no counterpart).  Parameters: one flat FP32 array of
 * ksc_mlp_n_params() values, W1[4][64] b1[64] W2[64][64] b2[64] W3[64][2] b3[2]
 * (row-major).  Inputs and targets are standardised inside the kernels with
 * the mean / standard deviation given to ksc_mlp_set_norm (default 0 / 1).
 * Loss: mean over samples and both outputs of the squared standardised error.
 */
typedef struct ksc_mlp ksc_mlp; /* opaque, library-owned */

int ksc_mlp_n_params(void);
/* New model with Glorot-uniform weights from a splitmix64 stream of `seed`,
 * zero biases, zero Adam state.  Synchronous.  Errors: ARG, NOMEM, CUDA. */
int ksc_mlp_create(unsigned long long seed, ksc_mlp **out);
/* Standardisation constants (host arrays of 4, 4, 2, 2 floats; std > 0). */
int ksc_mlp_set_norm(ksc_mlp *m, const float *x_mean, const float *x_std,
                     const float *y_mean, const float *y_std);
int ksc_mlp_get_params(const ksc_mlp *m, float *h_params);  /* synchronous */
int ksc_mlp_set_params(ksc_mlp *m, const float *h_params);  /* synchronous */
/* d_y[n][2] = model(d_x[n][4]) (device arrays, unstandardised units).
 * Asynchronous on `stream`. */
int ksc_mlp_predict(const ksc_mlp *m, const float *d_x, int n, float *d_y,
                    void *stream);
/* Gradient of the loss over the n samples (d_x[n][4], targets d_t[n][2],
 * device) with respect to the parameters, into h_grad[ksc_mlp_n_params()]
 * (host); *h_loss (may be NULL) receives the loss.  Synchronous (legacy
 * default stream). */
int ksc_mlp_grad(const ksc_mlp *m, const float *d_x, const float *d_t, int n,
                 float *h_grad, float *h_loss);
/* `epochs` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8, step size lr),
 * one epoch replayed as a CUDA graph on `stream`; *h_loss (may be NULL)
 * receives the loss evaluated in the last epoch (before its update), after
 * which the call has synchronised the stream. */
int ksc_mlp_train(ksc_mlp *m, const float *d_x, const float *d_t, int n,
                  int epochs, float lr, void *stream, float *h_loss);
/* Choose among n candidate splits h_x[n][4] (host): predicts on the GPU and
 * returns in *best the candidate of least cost among those whose predicted
 * log10 eps_C <= log10_bound - margin, or -1 if none.  The cost of a
 * candidate is max(predicted GPU time, h_host_ms[i]) -- the two halves of the
 * split run concurrently (Fig. 1) -- with h_host_ms (may be NULL: GPU time
 * only) the host cost of its harmonic half in ms (e.g. ksc_cost_eval's t_host
 * for the caller's host).  When it returns -1 the caller falls back to the
 * scan (ksc_scan_split), and a measured run of the chosen split decides.
 * h_pred (may be NULL) receives
 * the n x 2 predictions.  Synchronous. */
int ksc_mlp_select(const ksc_mlp *m, const float *h_x, int n, double log10_bound,
                   double margin, const double *h_host_ms, int *best, float *h_pred);
void ksc_mlp_free(ksc_mlp *m);

/* Release a split and its device memory (NULL is a no-op). */
void ksc_free_split(ksc_split *s);

/* Human-readable name of a status code. */
const char *ksc_status_string(int status);
/* Message of the last error on the calling thread ("" if none). */
const char *ksc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KSCONV_H */
